// mlba_api.cu — host runtime and C ABI of the MLBA library (include/mlba.h).
//
// A batch owns: a table of problem descriptors (Prob) and states (State) in
// device memory, one device arena holding every problem's buffers, and the
// item lists that map CTAs to (problem, block).  One step of the algorithm is
// a fixed sequence of batched launches captured once into a CUDA graph; each
// replay advances every live problem by one iteration.  A context for a
// single problem is a batch of one.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <new>
#include <string>

#include "../../include/mlba.h"
#include "mlba_internal.cuh"
#include "mlba_launch.h"

using namespace mlba;

namespace {

// graph nodes per iteration for the alpha_n solve: 1 bracketing pass and
// Halley passes (FP64 accepts only steps below its tighter tolerance)
template <typename T> constexpr int ns_passes() { return sizeof(T) == 8 ? 6 : 4; }
constexpr size_t ALIGN = 256;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return MLBA_E_CUDA;    \
  } while (0)

struct HostProb {
  Prob pd;                       // host copy with device pointers filled in
  std::vector<double> psf;       // p x p, the PSF used by A
  std::vector<double> psf_pre;   // PSF of the preconditioner (H or H~)
  std::vector<int> runs;         // (b, lo, hi, offset) per nonzero PSF column
  std::vector<double> rw;        // packed run weights H[lo..hi][b], then the same runs reversed
  std::vector<double> hy, hx;
  size_t off[NSLOT + 16];
};

struct ItemList {
  int2* dev = nullptr;
  int count = 0;
  int sec[2 * FRAME_SECTIONS] = {0};   // framelet list at L >= 3: (offset, count) per section
};

// The launches of one step over a set of problems.
struct StepLists {
  ItemList blur, corr, reblur, corr_kry, blur_kry, rows_spec, cols_stat, cols_ns, spec, rows_kry,
      cols_kry, vec_kry, vec_kry_bc, frame, ar_rows, ar_cols;
  // FFT blur path: forward (f) and adjoint (a) convolution entries, and the
  // epilogues on the problems (residual, correlation V, reblurring into U)
  ItemList fc_pad_f, fc_rows_f, fc_cols_f, fc_out_r, fc_pad_a, fc_rows_a, fc_cols_a, fc_out_v, fc_out_u;
  ItemList balance;   // balanced formulation: u <- f + u
  // (two-group graphs) the row passes of the stationary and of the 4-NS
  // problems apart, so that each kind's transform chain is one graph branch
  ItemList rows_st, rows_ns;
  int any_krylov = 0, any_spec = 0, any_ns = 0, any_ar = 0, pcg_max = 5;
};
struct StepItems {
  std::vector<int2> blur, corr, reblur, corr_kry, blur_kry, rows_spec, cols_stat, cols_ns, spec,
      rows_kry, cols_kry, vec_kry, vec_kry_bc, ar_rows, ar_cols;
  std::vector<int2> fc_pad_f, fc_rows_f, fc_cols_f, fc_out_r, fc_pad_a, fc_rows_a, fc_cols_a,
      fc_out_v, fc_out_u, balance;
  std::vector<int2> frame[FRAME_SECTIONS];   // see add_frame_items
  std::vector<int2> rows_st, rows_ns;
  int any_krylov = 0, any_spec = 0, any_ns = 0, any_ar = 0, pcg_max = 5;
};

// Framelet launches of problem i: levels <= 2, the tiles of the fused sweep
// (section 0); levels >= 3, the BC fold of the correlation (section 0, BC
// problems that apply A^T), the low-pass chain (section 1) and the level
// kernels of level L .. 1 (sections 2 ..).
void add_frame_items(const Prob& pd, int i, int levels, int shape,
                     std::vector<int2> (&fs)[FRAME_SECTIONS]) {
  auto add = [&](std::vector<int2>& L, int nblk) { for (int k = 0; k < nblk; ++k) L.push_back(make_int2(i, k)); };
  if (levels <= 2) { add(fs[0], frame_tiles(pd.nf, levels, shape)); return; }
  if (pd.use_adj && pd.bc != BC_RECT && pd.bc != BC_AR && !pd.balanced) add(fs[0], pd.nblk_vec);
  add(fs[1], lowpass_blocks(pd.nf));
  for (int k = 0; k < levels; ++k) add(fs[2 + k], lev_tiles(pd.nf, levels - k));
}

// parts of a step: a = residual and stop rule, then the preconditioner;
// b = A^T and the framelet update
enum { PART_A = 1, PART_B = 2, PART_ALL = 3 };

}  // namespace

struct mlba_batch {
  int dtype = MLBA_F32, z_store = MLBA_F32, levels = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<HostProb> hp;
  Prob* d_probs = nullptr;
  State* d_states = nullptr;
  State* d_opstates = nullptr;
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t zero_bytes = 0;        // [arena, arena + zero_bytes): every problem's f and z^0
  // item lists
  ItemList blur, corr, reblur, corr_kry, blur_kry, rows_spec, cols_stat, cols_ns, spec, rows_kry,
      cols_kry, vec_kry, vec_kry_bc, frame, corr_all, rows_all, cols_all, spec_all, vec_all,
      ar_rows, ar_cols;
  // FFT blur path (see StepLists); the *_all_f / *_all_a lists hold every
  // convolution entry and serve the operator entry points
  ItemList fc_pad_f, fc_rows_f, fc_cols_f, fc_out_r, fc_pad_a, fc_rows_a, fc_cols_a, fc_out_v, fc_out_u;
  std::vector<HostProb> fc;      // convolution entries, table indices count + k
  int blur_path = 0;
  ItemList balance;
  int formulation = 0;
  std::vector<int2*> allocs;
  size_t smem_stencil = 0, smem_fft = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool has_data = false;
  int any_krylov = 0, any_spec = 0, any_ns = 0, any_stat = 0, any_ar = 0;
  // Two-group schedule (batches of two or more problems): group 1 runs half a
  // step behind group 0 on a second stream, so that one group's framelet
  // sweep (HBM-bound) overlaps the other group's residual and preconditioner
  // (latency-bound).  iterate(k) replays: head (group 0: part a), body k - 1
  // times (group 0: part b, part a | group 1: part a, part b), tail (group 0:
  // part b | group 1: part a, part b); every problem then has done k steps.
  bool split = false;
  StepLists grp[2];
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // a parallel branch inside one step: the stationary column pass beside the
  // 4-NS chain (index 0 for the batch stream, 1 for the side stream)
  cudaStream_t br[2] = {nullptr, nullptr};
  cudaEvent_t ev_bf[2] = {nullptr, nullptr}, ev_bj[2] = {nullptr, nullptr};
  cudaGraph_t g_head = nullptr, g_body = nullptr, g_tail = nullptr;
  cudaGraphExec_t x_head = nullptr, x_body = nullptr, x_tail = nullptr;
  // framelet tile shape (k_frame.cu) and how it was chosen
  int frame_shape = 0;
  int frame_tuned = 0;          // 0 default, 1 measured here, 2 from the cache, 3 forced
  float frame_us = 0.f;         // measured time of one launch of the chosen shape
  // Persistent schedule (opts.persistent): the stage program of one step, the
  // barrier words, and the cooperative launch geometry (k_persist.cu)
  bool persistent = false;
  PersistStage* d_stages = nullptr;
  int nstages = 0;
  void* d_ctl = nullptr;
  int p_grid = 0, p_stencil_slot = 0, p_frame_slot = 0;
  size_t p_smem = 0;
  unsigned long long p_wait_ns = 1000000000ull;
  cudaGraph_t p_graph = nullptr;          // memset of the barrier words -> the kernel
  cudaGraphExec_t p_exec = nullptr;
  cudaGraphNode_t p_knode = nullptr;
  int p_k = 0;                            // step count the instantiated graph runs
};

struct mlba_ctx {
  mlba_batch* b;
};

namespace {

size_t tsize(int dtype) { return dtype == MLBA_F64 ? 8 : 4; }
size_t zsize(int zs) { return zs == MLBA_F64 ? 8 : (zs == MLBA_BF16 ? 2 : 4); }
size_t al(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// elements of the column-blocked spectrum (padding of the last block included)
int fft_pad(int i) { return i + (i >> 4); }   // shared-memory slot of element i (k_fft.cu)
size_t spec_elems(const Prob& pd) { return (size_t)pd.nblk_cols * pd.n * pd.cb; }
int vec_blocks(size_t elems) {
  return (int)((elems + VEC_THREADS * VEC_PER_THREAD - 1) / (VEC_THREADS * VEC_PER_THREAD));
}

// Radix passes of the length-n FFT: as many radix-16 passes as divide n, then
// at most one of 8, 4 or 2 for the rest of the power of two, then 3s and 5s,
// then every prime factor above 5 as a direct-sum pass (any n factors within
// MAX_STAGES passes: n <= 4096 has at most 12 prime factors).
bool fft_plan(Prob& pd) {
  int m = pd.nfft, s = 0;
  pd.nr16 = pd.r2 = pd.nr3 = pd.nr5 = pd.nrany = 0;
  while (m % 16 == 0 && s < MAX_STAGES) { pd.radix[s++] = 16; m /= 16; ++pd.nr16; }
  for (int r : {8, 4, 2})
    if (m % r == 0 && s < MAX_STAGES) { pd.radix[s++] = r; m /= r; pd.r2 = r; break; }
  while (m % 3 == 0 && s < MAX_STAGES) { pd.radix[s++] = 3; m /= 3; ++pd.nr3; }
  while (m % 5 == 0 && s < MAX_STAGES) { pd.radix[s++] = 5; m /= 5; ++pd.nr5; }
  for (int f = 7; m > 1 && s < MAX_STAGES;) {
    if ((long long)f * f > m) f = m;          // the rest is prime
    if (m % f == 0) { pd.radix[s++] = f; m /= f; ++pd.nrany; }
    else f += 2;
  }
  pd.nstage = s;
  return m == 1;
}

bool quad_symmetric(const std::vector<double>& h, int p) {
  double mx = 0;
  for (double v : h) mx = std::max(mx, std::fabs(v));
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      const double v = h[a * p + b];
      if (std::fabs(v - h[(p - 1 - a) * p + b]) > 1e-14 * mx) return false;
      if (std::fabs(v - h[a * p + (p - 1 - b)]) > 1e-14 * mx) return false;
    }
  return true;
}

// H~ of Section 4.3, each quadrant orbit computed once so the result is
// exactly symmetric
std::vector<double> symmetrized(const std::vector<double>& h, int p) {
  std::vector<double> s(h.size());
  for (int a = 0; a <= (p - 1) / 2; ++a)
    for (int b = 0; b <= (p - 1) / 2; ++b) {
      const int a2 = p - 1 - a, b2 = p - 1 - b;
      const double v = 0.25 * (h[a * p + b] + h[a2 * p + b] + h[a * p + b2] + h[a2 * p + b2]);
      s[a * p + b] = s[a2 * p + b] = s[a * p + b2] = s[a2 * p + b2] = v;
    }
  return s;
}

bool rank_one(const std::vector<double>& h, int p, std::vector<double>& u, std::vector<double>& v) {
  int a0 = 0, b0 = 0;
  double mx = 0;
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b)
      if (std::fabs(h[a * p + b]) > mx) { mx = std::fabs(h[a * p + b]); a0 = a; b0 = b; }
  if (mx == 0) return false;
  u.assign(p, 0); v.assign(p, 0);
  for (int a = 0; a < p; ++a) u[a] = h[a * p + b0];
  for (int b = 0; b < p; ++b) v[b] = h[a0 * p + b] / h[a0 * p + b0];
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b)
      if (std::fabs(h[a * p + b] - u[a] * v[b]) > 1e-14 * mx) return false;
  return true;
}

template <typename T>
void put(unsigned char* host, size_t off, const std::vector<double>& v) {
  T* d = reinterpret_cast<T*>(host + off);
  for (size_t i = 0; i < v.size(); ++i) d[i] = (T)v[i];
}

int build_list(mlba_batch* B, ItemList& L, const std::vector<int2>& items) {
  L.count = (int)items.size();
  if (L.count == 0) return MLBA_OK;
  CK(cudaMalloc(&L.dev, items.size() * sizeof(int2)));
  B->allocs.push_back(L.dev);
  CK(cudaMemcpy(L.dev, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
  return MLBA_OK;
}

int build_fc_lists(mlba_batch* B, StepLists& L, const StepItems& v) {
  int rc = MLBA_OK;
  rc |= build_list(B, L.fc_pad_f, v.fc_pad_f); rc |= build_list(B, L.fc_rows_f, v.fc_rows_f);
  rc |= build_list(B, L.fc_cols_f, v.fc_cols_f); rc |= build_list(B, L.fc_out_r, v.fc_out_r);
  rc |= build_list(B, L.fc_pad_a, v.fc_pad_a); rc |= build_list(B, L.fc_rows_a, v.fc_rows_a);
  rc |= build_list(B, L.fc_cols_a, v.fc_cols_a); rc |= build_list(B, L.fc_out_v, v.fc_out_v);
  rc |= build_list(B, L.fc_out_u, v.fc_out_u);
  return rc;
}

// the framelet list: one section (levels <= 2) or the sections concatenated
int build_frame_list(mlba_batch* B, ItemList& L, const std::vector<int2> (&fs)[FRAME_SECTIONS],
                     int levels) {
  if (levels <= 2) return build_list(B, L, fs[0]);
  std::vector<int2> all;
  for (int k = 0; k < 2 + levels; ++k) {
    L.sec[2 * k] = (int)all.size();
    L.sec[2 * k + 1] = (int)fs[k].size();
    all.insert(all.end(), fs[k].begin(), fs[k].end());
  }
  const int rc = build_list(B, L, all);
  return rc;
}

State initial_state(const Prob& pd) {
  State s;
  std::memset(&s, 0, sizeof(s));
  s.stop_iter = -1;
  s.alpha_n = pd.alpha;
  s.nb = 0.0;
  return s;
}

template <typename T, typename TZ>
void enqueue_step(mlba_batch* B, const StepLists& L, int part, cudaStream_t s) {
  const Prob* P = B->d_probs;
  State* S = B->d_states;
  if (part & PART_A) {
    // a2: r = g - A f with ||r||^2 and the stop rule
    launch_stencil<T>(ST_FWD_RESID, P, S, L.blur.dev, L.blur.count, SL_F, SL_R, SL_G, 0,
                      B->smem_stencil, s);
    // (FFT blur path: f extended by the BCs, A f by convolution with the PSF)
    if (L.fc_out_r.count) {
      launch_fc_pad<T>(P, S, L.fc_pad_f.dev, L.fc_pad_f.count, 0, -1, s);
      launch_rows_fwd<T>(P, S, L.fc_rows_f.dev, L.fc_rows_f.count, SL_R, 0, B->smem_fft, s);
      launch_cols<T>(P, S, L.fc_cols_f.dev, L.fc_cols_f.count, COL_OP, 0, 1.0, W_TIKH, B->smem_fft, s);
      launch_rows_inv<T>(P, S, L.fc_rows_f.dev, L.fc_rows_f.count, SL_T, 0, B->smem_fft, s);
      launch_fc_out<T>(P, S, L.fc_out_r.dev, L.fc_out_r.count, FC_RESID_MODE, 0, SL_R, s);
    }
    // a4: spectral preconditioners (Algorithms 1, 3, 4, 4-NS)
    const int bs = (s == B->stream) ? 0 : (s == B->side ? 1 : -1);
    if (L.any_spec && L.rows_st.count > 0 && L.rows_ns.count > 0 && bs >= 0 && B->br[bs] != nullptr) {
      // Stationary and 4-NS problems both present (two-group graphs): each
      // kind's transform chain is one branch of the graph; they touch
      // disjoint problems, so their partial waves overlap throughout
      cudaStream_t sb = B->br[bs];
      cudaEventRecord(B->ev_bf[bs], s);
      cudaStreamWaitEvent(sb, B->ev_bf[bs], 0);
      launch_rows_fwd<T>(P, S, L.rows_st.dev, L.rows_st.count, SL_R, 0, B->smem_fft, sb);
      launch_cols<T>(P, S, L.cols_stat.dev, L.cols_stat.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, sb);
      launch_rows_inv<T>(P, S, L.rows_st.dev, L.rows_st.count, SL_T, 0, B->smem_fft, sb);
      cudaEventRecord(B->ev_bj[bs], sb);
      launch_rows_fwd<T>(P, S, L.rows_ns.dev, L.rows_ns.count, SL_R, 0, B->smem_fft, s);
      launch_cols<T>(P, S, L.cols_ns.dev, L.cols_ns.count, COL_FWD, 0, 0.0, 0, B->smem_fft, s);
      for (int k = 1; k < ns_passes<T>(); ++k) launch_spec<T>(P, S, L.spec.dev, L.spec.count, 0, s);
      launch_cols<T>(P, S, L.cols_ns.dev, L.cols_ns.count, COL_NS_INV, 0, 0.0, 0, B->smem_fft, s);
      launch_rows_inv<T>(P, S, L.rows_ns.dev, L.rows_ns.count, SL_T, 0, B->smem_fft, s);
      cudaStreamWaitEvent(s, B->ev_bj[bs], 0);
    } else if (L.any_spec) {
      launch_rows_fwd<T>(P, S, L.rows_spec.dev, L.rows_spec.count, SL_R, 0, B->smem_fft, s);
      // The stationary column pass and the 4-NS chain (forward pass with the
      // bracketing sums, Halley passes, weighted inverse) work on disjoint
      // problems: with both present the stationary pass runs as a parallel
      // branch, so that the partial waves of the two launches overlap.
      const int bi = (s == B->stream) ? 0 : (s == B->side ? 1 : -1);
      const bool fork = L.any_ns && L.cols_stat.count > 0 && bi >= 0 && B->br[bi] != nullptr;
      cudaStream_t sc = s;
      if (fork) {
        cudaEventRecord(B->ev_bf[bi], s);
        cudaStreamWaitEvent(B->br[bi], B->ev_bf[bi], 0);
        sc = B->br[bi];
      }
      launch_cols<T>(P, S, L.cols_stat.dev, L.cols_stat.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, sc);
      if (fork) cudaEventRecord(B->ev_bj[bi], sc);
      if (L.any_ns) {
        launch_cols<T>(P, S, L.cols_ns.dev, L.cols_ns.count, COL_FWD, 0, 0.0, 0, B->smem_fft, s);
        // (the bracketing pass runs inside the forward column pass)
        for (int k = 1; k < ns_passes<T>(); ++k) launch_spec<T>(P, S, L.spec.dev, L.spec.count, 0, s);
        launch_cols<T>(P, S, L.cols_ns.dev, L.cols_ns.count, COL_NS_INV, 0, 0.0, 0, B->smem_fft, s);
      }
      if (fork) cudaStreamWaitEvent(s, B->ev_bj[bi], 0);
      launch_rows_inv<T>(P, S, L.rows_spec.dev, L.rows_spec.count, SL_T, 0, B->smem_fft, s);
    }
    // a4 with the antireflective transform (Algorithms 1, 3, 4 on antireflective A)
    if (L.any_ar) {
      launch_ar_rows<T>(P, S, L.ar_rows.dev, L.ar_rows.count, SL_R, 0, 0, B->smem_fft, s);
      launch_ar_cols<T>(P, S, L.ar_cols.dev, L.ar_cols.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, s);
      launch_ar_rows<T>(P, S, L.ar_rows.dev, L.ar_rows.count, SL_T, 1, 0, B->smem_fft, s);
    }
    // a4': Algorithm 2, PCG on (A A^T + alpha I) t = r preconditioned by (CC^T + alpha I)^{-1}
    if (L.any_krylov) {
      const int maxs = L.pcg_max;
      launch_vec<T>(VEC_PCG_INIT, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
      launch_rows_fwd<T>(P, S, L.rows_kry.dev, L.rows_kry.count, SL_PRES, 1, B->smem_fft, s);
      launch_cols<T>(P, S, L.cols_kry.dev, L.cols_kry.count, COL_FUSED, 1, 0.0, 0, B->smem_fft, s);
      launch_rows_inv<T>(P, S, L.rows_kry.dev, L.rows_kry.count, SL_PZ, 1, B->smem_fft, s);
      launch_vec<T>(VEC_PCG_RHO0, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
      for (int k = 0; k < maxs; ++k) {
        launch_stencil<T>(ST_CORR, P, S, L.corr_kry.dev, L.corr_kry.count, SL_PP, SL_V, SL_V, 1,
                          B->smem_stencil, s);
        launch_vec<T>(VEC_FOLD, P, S, L.vec_kry_bc.dev, L.vec_kry_bc.count, 1, s);
        launch_stencil<T>(ST_FWD_PCGQ, P, S, L.blur_kry.dev, L.blur_kry.count, -1, SL_PQ, SL_PP, 1,
                          B->smem_stencil, s);
        launch_vec<T>(VEC_PCG_AXPY, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
        launch_rows_fwd<T>(P, S, L.rows_kry.dev, L.rows_kry.count, SL_PRES, 1, B->smem_fft, s);
        launch_cols<T>(P, S, L.cols_kry.dev, L.cols_kry.count, COL_FUSED, 1, 0.0, 0, B->smem_fft, s);
        launch_rows_inv<T>(P, S, L.rows_kry.dev, L.rows_kry.count, SL_PZ, 1, B->smem_fft, s);
        launch_vec<T>(VEC_PCG_RHO, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
        launch_vec<T>(VEC_PCG_PUPD, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
      }
      launch_vec<T>(VEC_PCG_FINISH, P, S, L.vec_kry.dev, L.vec_kry.count, 1, s);
    }
  }
  if (part & PART_B) {
    // a6: full correlation of t (A^T up to the BC fold); antireflective BCs:
    // the reblurring A' t into U
    launch_stencil<T>(ST_CORR, P, S, L.corr.dev, L.corr.count, -1, SL_V, SL_V, 0, B->smem_stencil, s);
    launch_stencil<T>(ST_REBLUR, P, S, L.reblur.dev, L.reblur.count, -1, -1, SL_U, 0, B->smem_stencil, s);
    // (FFT blur path: t placed at (c, c), or extended antireflectively, and
    // correlated with the PSF)
    if (L.fc_pad_a.count) {
      launch_fc_pad<T>(P, S, L.fc_pad_a.dev, L.fc_pad_a.count, 1, -1, s);
      launch_rows_fwd<T>(P, S, L.fc_rows_a.dev, L.fc_rows_a.count, SL_R, 0, B->smem_fft, s);
      launch_cols<T>(P, S, L.fc_cols_a.dev, L.fc_cols_a.count, COL_OP, 0, 1.0, W_TIKH, B->smem_fft, s);
      launch_rows_inv<T>(P, S, L.fc_rows_a.dev, L.fc_rows_a.count, SL_T, 0, B->smem_fft, s);
      launch_fc_out<T>(P, S, L.fc_out_v.dev, L.fc_out_v.count, FC_CORR_MODE, 1, SL_V, s);
      launch_fc_out<T>(P, S, L.fc_out_u.dev, L.fc_out_u.count, FC_STORE_MODE, 1, SL_U, s);
    }
    // balanced formulation: x = S_mu(W (f + u))
    launch_balance<T>(P, S, L.balance.dev, L.balance.count, s);
    // a1: z += W u, x = S_mu(z), f = W^T x
    launch_frame<T, TZ>(P, S, L.frame.dev, L.frame.count, L.frame.sec, -1, SL_F, nullptr, nullptr,
                        0.0, B->levels, B->frame_shape, s);
  }
}

void enqueue_dispatch(mlba_batch* B, const StepLists& L, int part, cudaStream_t s) {
  if (B->dtype == MLBA_F64) enqueue_step<double, double>(B, L, part, s);
  else if (B->z_store == MLBA_BF16) enqueue_step<float, __nv_bfloat16>(B, L, part, s);
  else enqueue_step<float, float>(B, L, part, s);
}

StepLists all_lists(const mlba_batch* B) {
  StepLists L;
  L.blur = B->blur; L.corr = B->corr; L.reblur = B->reblur; L.corr_kry = B->corr_kry; L.blur_kry = B->blur_kry;
  L.rows_spec = B->rows_spec; L.cols_stat = B->cols_stat; L.cols_ns = B->cols_ns; L.spec = B->spec;
  L.rows_kry = B->rows_kry; L.cols_kry = B->cols_kry; L.vec_kry = B->vec_kry;
  L.vec_kry_bc = B->vec_kry_bc; L.frame = B->frame;
  L.any_krylov = B->any_krylov; L.any_spec = B->any_spec; L.any_ns = B->any_ns;
  L.ar_rows = B->ar_rows; L.ar_cols = B->ar_cols; L.any_ar = B->any_ar;
  L.fc_pad_f = B->fc_pad_f; L.fc_rows_f = B->fc_rows_f; L.fc_cols_f = B->fc_cols_f;
  L.fc_out_r = B->fc_out_r; L.fc_pad_a = B->fc_pad_a; L.fc_rows_a = B->fc_rows_a;
  L.fc_cols_a = B->fc_cols_a; L.fc_out_v = B->fc_out_v; L.fc_out_u = B->fc_out_u;
  L.balance = B->balance;
  L.pcg_max = B->hp.empty() ? 5 : B->hp[0].pd.pcg_max;
  return L;
}

// the launches of one step of problem i (kinds as in the whole-batch lists)
// The FFT-blur-path launches of problem i (pd.fc set): its forward and
// adjoint convolution entries sf, sa (their own geometry), and the epilogues
void collect_fc(const Prob& pd, int i, const Prob& sf, const Prob& sa, StepItems& V) {
  auto addk = [&](std::vector<int2>& L, int x, int nblk) { for (int k = 0; k < nblk; ++k) L.push_back(make_int2(x, k)); };
  const int fi = pd.fc_sh[0], ai = pd.fc_sh[1];
  addk(V.fc_pad_f, fi, sf.nblk_vec); addk(V.fc_rows_f, fi, sf.nblk_rows); addk(V.fc_cols_f, fi, sf.nblk_cols);
  addk(V.fc_out_r, i, pd.nblk_vec);
  if (pd.use_adj) {
    addk(V.fc_pad_a, ai, sa.nblk_vec); addk(V.fc_rows_a, ai, sa.nblk_rows); addk(V.fc_cols_a, ai, sa.nblk_cols);
    if (pd.bc == BC_AR) addk(V.fc_out_u, i, pd.nblk_vec);
    else addk(V.fc_out_v, i, vec_blocks((size_t)pd.ne * pd.ne));
  }
}

void collect_step(const Prob& pd, int i, int levels, int shape, StepItems& V) {
  auto add = [&](std::vector<int2>& L, int nblk) { for (int k = 0; k < nblk; ++k) L.push_back(make_int2(i, k)); };
  if (!pd.fc) add(V.blur, pd.nblk_blur);
  add_frame_items(pd, i, levels, shape, V.frame);
  if (pd.use_adj && !pd.fc) {
    if (pd.bc == BC_AR) add(V.reblur, pd.nblk_blur);
    else add(V.corr, pd.nblk_corr);
  }
  if (pd.balanced) add(V.balance, vec_blocks((size_t)pd.nf * pd.nf));
  const bool specp = pd.transform != TR_NONE;
  if (pd.precond == P_KRYLOV) {
    add(V.corr_kry, pd.nblk_corr); add(V.blur_kry, pd.nblk_blur); add(V.rows_kry, pd.nblk_rows);
    add(V.cols_kry, pd.nblk_cols); add(V.vec_kry, pd.nblk_vec);
    if (pd.bc != BC_RECT) add(V.vec_kry_bc, pd.nblk_vec);
    V.any_krylov = 1;
  } else if (pd.transform == TR_AR) {
    add(V.ar_rows, pd.nblk_rows); add(V.ar_cols, pd.nblk_cols);
    V.any_ar = 1;
  } else if (specp) {
    add(V.rows_spec, pd.nblk_rows);
    V.any_spec = 1;
    if (pd.ns) {
      add(V.rows_ns, pd.nblk_rows); add(V.cols_ns, pd.nblk_cols); add(V.spec, pd.nblk_spec);
      V.any_ns = 1;
    } else {
      add(V.rows_st, pd.nblk_rows); add(V.cols_stat, pd.nblk_cols);
    }
  }
  V.pcg_max = pd.pcg_max;
}

// Low priority for the framelet launches of the two-group graphs: the
// latency-bound launches of the other group take SM resources first and the
// framelet sweep fills the rest.
int set_node_priorities(cudaGraph_t g, int lo, int hi) {
  size_t cnt = 0;
  CK(cudaGraphGetNodes(g, nullptr, &cnt));
  std::vector<cudaGraphNode_t> nodes(cnt);
  CK(cudaGraphGetNodes(g, nodes.data(), &cnt));
  for (size_t i = 0; i < cnt; ++i) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nodes[i], &t));
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    CK(cudaGraphKernelNodeGetParams(nodes[i], &kp));
    cudaKernelNodeAttrValue v;
    std::memset(&v, 0, sizeof(v));
    v.priority = is_frame_kernel(kp.func) ? lo : hi;
    CK(cudaGraphKernelNodeSetAttribute(nodes[i], cudaKernelNodeAttributePriority, &v));
  }
  return MLBA_OK;
}

// capture parts pa of group 0 and pb of group 1 (0: none) as one graph; the
// group-0 parts run in order a, b (head) or b, a (body) on the batch stream,
// the group-1 parts (a then b) on the side stream
int capture_split(mlba_batch* B, int pa, bool b_first, int pb, cudaGraph_t* g, cudaGraphExec_t* x) {
  cudaStream_t s = B->stream;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MLBA_E_CUDA;
  if (pb) {
    cudaEventRecord(B->ev_fork, s);
    cudaStreamWaitEvent(B->side, B->ev_fork, 0);
    if (pb & PART_A) enqueue_dispatch(B, B->grp[1], PART_A, B->side);
    if (pb & PART_B) enqueue_dispatch(B, B->grp[1], PART_B, B->side);
  }
  if (b_first) {
    if (pa & PART_B) enqueue_dispatch(B, B->grp[0], PART_B, s);
    if (pa & PART_A) enqueue_dispatch(B, B->grp[0], PART_A, s);
  } else {
    if (pa & PART_A) enqueue_dispatch(B, B->grp[0], PART_A, s);
    if (pa & PART_B) enqueue_dispatch(B, B->grp[0], PART_B, s);
  }
  if (pb) {
    cudaEventRecord(B->ev_join, B->side);
    cudaStreamWaitEvent(s, B->ev_join, 0);
  }
  if (cudaStreamEndCapture(s, g) != cudaSuccess) return MLBA_E_CUDA;
  int lo = 0, hi = 0;
  CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (set_node_priorities(*g, lo, hi) != MLBA_OK) return MLBA_E_CUDA;
  CK(cudaGraphInstantiate(x, *g, 0));
  return MLBA_OK;
}

// Split the problems into two groups of about equal work (largest first, each
// to the lighter group) and capture the head, body and tail graphs.
int build_split(mlba_batch* B) {
  const int count = (int)B->hp.size();
  if (count < 2) return MLBA_OK;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto work = [&](int i) { const Prob& pd = B->hp[i].pd; return (double)pd.nf * pd.nf; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<int> grp(count, 0);
  double w[2] = {0.0, 0.0};
  for (int i : order) { const int g = w[1] < w[0] ? 1 : 0; grp[i] = g; w[g] += work(i); }
  StepItems V[2];
  for (int i = 0; i < count; ++i) {
    const Prob& pd = B->hp[i].pd;
    collect_step(pd, i, B->levels, B->frame_shape, V[grp[i]]);
    if (pd.fc)
      collect_fc(pd, i, B->fc[pd.fc_sh[0] - count].pd, B->fc[pd.fc_sh[1] - count].pd, V[grp[i]]);
  }
  int rc = MLBA_OK;
  for (int g = 0; g < 2; ++g) {
    StepLists& L = B->grp[g];
    const StepItems& v = V[g];
    rc |= build_list(B, L.blur, v.blur); rc |= build_list(B, L.corr, v.corr);
    rc |= build_list(B, L.reblur, v.reblur);
    rc |= build_list(B, L.corr_kry, v.corr_kry); rc |= build_list(B, L.blur_kry, v.blur_kry);
    rc |= build_list(B, L.rows_spec, v.rows_spec); rc |= build_list(B, L.cols_stat, v.cols_stat);
    rc |= build_list(B, L.cols_ns, v.cols_ns); rc |= build_list(B, L.spec, v.spec);
    rc |= build_list(B, L.rows_st, v.rows_st); rc |= build_list(B, L.rows_ns, v.rows_ns);
    rc |= build_list(B, L.rows_kry, v.rows_kry); rc |= build_list(B, L.cols_kry, v.cols_kry);
    rc |= build_list(B, L.vec_kry, v.vec_kry); rc |= build_list(B, L.vec_kry_bc, v.vec_kry_bc);
    rc |= build_frame_list(B, L.frame, v.frame, B->levels);
    rc |= build_list(B, L.ar_rows, v.ar_rows); rc |= build_list(B, L.ar_cols, v.ar_cols);
    rc |= build_fc_lists(B, L, v);
    rc |= build_list(B, L.balance, v.balance);
    L.any_krylov = v.any_krylov; L.any_spec = v.any_spec; L.any_ns = v.any_ns; L.any_ar = v.any_ar;
    L.pcg_max = B->hp[0].pd.pcg_max;
  }
  if (rc != MLBA_OK) return MLBA_E_CUDA;
  CK(cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming));
  if (capture_split(B, PART_A, false, 0, &B->g_head, &B->x_head) != MLBA_OK ||
      capture_split(B, PART_ALL, true, PART_ALL, &B->g_body, &B->x_body) != MLBA_OK ||
      capture_split(B, PART_B, false, PART_ALL, &B->g_tail, &B->x_tail) != MLBA_OK)
    return MLBA_E_CUDA;
  B->split = true;
  return MLBA_OK;
}

int set_smem_attrs(mlba_batch* B) {
  if (B->dtype == MLBA_F64) {
    CK(stencil_set_smem<double>(B->smem_stencil));
    CK(fft_set_smem<double>(B->smem_fft));
    CK((frame_set_smem<double, double>()));
  } else {
    CK(stencil_set_smem<float>(B->smem_stencil));
    CK(fft_set_smem<float>(B->smem_fft));
    if (B->z_store == MLBA_BF16) CK((frame_set_smem<float, __nv_bfloat16>()));
    else CK((frame_set_smem<float, float>()));
  }
  return MLBA_OK;
}

void frame_shape_of(const mlba_batch* B, int* tx, int* ty, int* pf) {
  frame_shape(B->frame_shape, tx, ty, pf);
}

void destroy_batch(mlba_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (cudaGraphExec_t x : {B->x_head, B->x_body, B->x_tail}) if (x) cudaGraphExecDestroy(x);
  for (cudaGraph_t g : {B->g_head, B->g_body, B->g_tail}) if (g) cudaGraphDestroy(g);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  if (B->side) cudaStreamDestroy(B->side);
  for (int q = 0; q < 2; ++q) {
    if (B->br[q]) cudaStreamDestroy(B->br[q]);
    if (B->ev_bf[q]) cudaEventDestroy(B->ev_bf[q]);
    if (B->ev_bj[q]) cudaEventDestroy(B->ev_bj[q]);
  }
  for (int2* p : B->allocs) cudaFree(p);
  if (B->arena) cudaFree(B->arena);
  if (B->d_probs) cudaFree(B->d_probs);
  if (B->d_states) cudaFree(B->d_states);
  if (B->d_opstates) cudaFree(B->d_opstates);
  if (B->p_exec) cudaGraphExecDestroy(B->p_exec);
  if (B->p_graph) cudaGraphDestroy(B->p_graph);
  if (B->d_stages) cudaFree(B->d_stages);
  if (B->d_ctl) cudaFree(B->d_ctl);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

// Launch geometry of the transform passes of a length-n problem (FFT length
// pd.nfft): transforms per CTA and the column blocking of the spectrum.
void transform_geometry(Prob& pd) {
  const int n = pd.n;
  const int cap = TR_CAP / std::max(pd.nfft, n);      // transforms per CTA
  const int pairs = (n + 1) / 2;
  {
    const int nb = (pairs + cap - 1) / cap;            // row CTAs, then pairs spread evenly
    pd.row_g = std::max(1, (pairs + nb - 1) / nb);
    pd.nblk_rows = (pairs + pd.row_g - 1) / pd.row_g;
  }
  {
    // column blocks: as few as the cap allows, then as even as possible
    // (real spectra, DCT and antireflective, move real columns in pairs)
    const bool dct = pd.transform == TR_DCT || pd.transform == TR_AR;
    const int units = dct ? pairs : pd.half;           // complex columns to transform
    const int nb = (units + cap - 1) / cap;
    pd.col_g = std::max(1, (units + nb - 1) / nb);
    pd.cb = dct ? 2 * pd.col_g : pd.col_g;
    pd.nblk_cols = ((dct ? n : pd.half) + pd.cb - 1) / pd.cb;
  }
  pd.nblk_spec = (int)((spec_elems(pd) + SPEC_THREADS * SPEC_PER_THREAD - 1) /
                       (SPEC_THREADS * SPEC_PER_THREAD));
}

// smallest 2^a 3^b 5^c >= m (fast radix passes for the convolution size)
int smooth_at_least(int m) {
  for (int x = m;; ++x) {
    int y = x;
    for (int f : {2, 3, 5}) while (y % f == 0) y /= f;
    if (y == 1) return x;
  }
}

// A convolution entry of problem `owner` (FFT blur path): an M x M DFT
// "problem" whose spectrum is the DFT of the PSF rotated by 180 degrees
// (forward: the column pass's conj(lambda) is then H^, convolution) or of
// the PSF itself (adjoint: conj(H^), correlation).
bool setup_conv_entry(const HostProb& own, int owner, int adj, HostProb& h) {
  const Prob& op = own.pd;
  Prob& pd = h.pd;
  std::memset(&pd, 0, sizeof(pd));
  const int M = smooth_at_least(op.ne);
  if (M > TR_CAP) return false;
  pd.n = pd.nf = pd.ne = M; pd.p = op.p; pd.c = op.c; pd.half = M / 2 + 1;
  pd.transform = TR_DFT; pd.precond = P_BCCB; pd.bc = BC_PERIODIC;
  pd.levels = op.levels; pd.nbands = op.nbands;
  pd.alpha = 1.0; pd.max_iter = -1; pd.sidx = owner;
  pd.nfft = M;
  if (!fft_plan(pd)) return false;
  transform_geometry(pd);
  pd.nblk_vec = vec_blocks((size_t)M * M);
  const int p = op.p;
  h.psf_pre.resize((size_t)p * p);
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b)
      h.psf_pre[(size_t)a * p + b] = adj ? own.psf[(size_t)a * p + b]
                                         : own.psf[(size_t)(p - 1 - a) * p + (p - 1 - b)];
  return true;
}

// Validate one problem and fill its host description (no device work).
int setup_problem(const mlba_problem& in, const mlba_opts& o, HostProb& h) {
  const int p = in.p, n = in.n;
  if (!in.psf || p < 1 || (p % 2) == 0 || n < p || n < 2) return MLBA_E_INVAL;
  if (p > MLBA_MAX_P) return MLBA_E_UNSUPPORTED;
  if (in.bc < 0 || in.bc > 4 || in.precond < 0 || in.precond > 5) return MLBA_E_INVAL;
  // antireflective BCs: Algorithm 2 is of no use there (Example 4)
  if (in.bc == MLBA_BC_ANTIREFLECTIVE && in.precond == MLBA_P_KRYLOV) return MLBA_E_INVAL;
  if (o.levels < 1 || o.levels > 4) return MLBA_E_INVAL;
  if (!(in.delta >= 0.0) || !(in.mu >= 0.0)) return MLBA_E_INVAL;
  const bool ns = in.precond == MLBA_P_TIKH_NS;
  if (in.bc == MLBA_RECT && (in.precond == MLBA_P_TIKH || (ns && !o.rect_ns_hybrid)))
    return MLBA_E_INVAL;   // Section 5: Algorithm 4 needs a square A
  if (!ns && in.precond != MLBA_P_NONE && !(in.alpha > 0.0)) return MLBA_E_INVAL;
  if (ns && in.bc == MLBA_RECT && !(in.alpha > 0.0)) return MLBA_E_INVAL;
  if (ns && !(in.delta > 0.0)) return MLBA_E_INVAL;
  if (!(o.q > 2.0 * o.rho && o.q < 1.0 && o.rho > 0.0 && o.rho < 0.5) && ns) return MLBA_E_INVAL;
  h.psf.assign(in.psf, in.psf + (size_t)p * p);
  for (double v : h.psf)
    if (!std::isfinite(v)) return MLBA_E_INVAL;
  Prob& pd = h.pd;
  std::memset(&pd, 0, sizeof(pd));
  pd.n = n; pd.p = p; pd.c = (p - 1) / 2;
  pd.nf = in.bc == MLBA_RECT ? n + p - 1 : n;
  pd.ne = n + p - 1;
  pd.half = n / 2 + 1;
  pd.bc = in.bc; pd.precond = in.precond; pd.levels = o.levels; pd.nbands = 8 * o.levels + 1;
  pd.ns = ns ? 1 : 0;
  pd.balanced = o.formulation == 1 ? 1 : 0;
  pd.use_adj = (in.precond == MLBA_P_TIKH || (ns && in.bc != MLBA_RECT)) ? 0 : 1;
  pd.max_iter = in.max_iter > 0 ? in.max_iter : o.max_iter;
  pd.stop = o.stop;
  pd.pcg_max = o.pcg_max;
  pd.mu = in.mu; pd.alpha = in.alpha; pd.gamma = o.gamma; pd.delta = in.delta;
  pd.q = o.q; pd.rho = o.rho; pd.tau = (1.0 + 2.0 * o.rho) / (1.0 - 2.0 * o.rho);
  pd.pcg_tol = o.pcg_tol;
  // transform (Section 4.1 / 4.3)
  const bool ar_bc = in.bc == MLBA_BC_ANTIREFLECTIVE;
  if (in.transform < 0 || in.transform > 3) return MLBA_E_INVAL;
  if (in.precond == MLBA_P_NONE) {
    pd.transform = TR_NONE;
  } else if (in.precond == MLBA_P_SYM) {
    // Section 4.3: Q from H~ under reflective BCs (DCT), or under
    // antireflective BCs for an antireflective A (antireflective transform)
    pd.transform = ar_bc ? TR_AR : TR_DCT;
    h.psf_pre = symmetrized(h.psf, p);
  } else {
    const int tr = in.transform;
    const bool sym = quad_symmetric(h.psf, p);
    if ((tr == MLBA_TR_DCT || tr == MLBA_TR_AR) && !sym) return MLBA_E_INVAL;
    // AUTO: periodic A is its own BCCB matrix (DFT); antireflective A is
    // diagonalised by the antireflective transform for a quadrantally
    // symmetric PSF (C = A) outside 4-NS, else the BCCB C as Examples 3 and 4
    // do; otherwise the reflective (DCT) matrix for a quadrantally symmetric
    // PSF, the periodic one if not
    int autotr;
    if (in.bc == MLBA_BC_PERIODIC) autotr = TR_DFT;
    else if (ar_bc) autotr = (sym && !ns) ? TR_AR : TR_DFT;
    else autotr = sym ? TR_DCT : TR_DFT;
    pd.transform = (tr == MLBA_TR_DFT) ? TR_DFT
                 : (tr == MLBA_TR_DCT ? TR_DCT : (tr == MLBA_TR_AR ? TR_AR : autotr));
    h.psf_pre = h.psf;
  }
  // the antireflective transform serves antireflective A outside 4-NS (it is
  // not unitary, Eq. Alg4_rev_7 is solved with spectral sums) and Algorithm 2
  if (pd.transform == TR_AR && (!ar_bc || ns || in.precond == MLBA_P_KRYLOV)) return MLBA_E_INVAL;
  pd.nfft = (pd.transform == TR_AR) ? 2 * (n - 1) : n;   // DST-I of n - 2 as a DFT of 2(n - 1)
  if (pd.transform != TR_NONE) {
    if (!fft_plan(pd)) return MLBA_E_UNSUPPORTED;
    // one transform must fit the per-CTA value budget of the smem FFT
    if (pd.nfft > TR_CAP || (pd.transform == TR_AR && n < 3)) return MLBA_E_UNSUPPORTED;
  }
  // taps: per PSF column the dense run of rows between its first and last
  // nonzero entry
  pd.ntaps = 0;
  for (int b = 0; b < p; ++b) {
    int lo = -1, hi = -1;
    for (int a = 0; a < p; ++a)
      if (h.psf[a * p + b] != 0.0) { if (lo < 0) lo = a; hi = a; ++pd.ntaps; }
    if (lo < 0) continue;
    h.runs.insert(h.runs.end(), {b, lo, hi, (int)h.rw.size()});
    for (int a = lo; a <= hi; ++a) h.rw.push_back(h.psf[a * p + b]);
  }
  if (pd.ntaps == 0) return MLBA_E_INVAL;
  pd.nruns = (int)h.runs.size() / 4;
  pd.nrw = (int)h.rw.size();
  // second copy with every run reversed (the order the forward stencil
  // consumes), so that a CTA copies its weights with one flat loop
  for (int r = 0; r < pd.nruns; ++r) {
    const int lo = h.runs[4 * r + 1], hi = h.runs[4 * r + 2], off = h.runs[4 * r + 3];
    for (int t = 0; t <= hi - lo; ++t) {
      const double v = h.rw[off + (hi - lo) - t];
      h.rw.push_back(v);
    }
  }
  pd.sep = rank_one(h.psf, p, h.hy, h.hx) && p > 1 ? 1 : 0;
  // launch geometry
  pd.nblk_blur = stencil_tiles(n);
  pd.nblk_corr = stencil_tiles(pd.ne);
  // the frame kernel indexes a z array (all bands) with 32-bit offsets
  if ((double)pd.nbands * pd.nf * pd.nf >= 2147483647.0) return MLBA_E_UNSUPPORTED;
  transform_geometry(pd);
  pd.nblk_vec = vec_blocks((size_t)n * n);
  return MLBA_OK;
}

// Build the spectrum of C / Q in FP64 on the device (Section 4.1).
int build_spectrum(mlba_batch* B, HostProb& h) {
  Prob& pd = h.pd;
  const int n = pd.n, p = pd.p, c = pd.c, half = pd.half;
  const bool dct = pd.transform == TR_DCT;
  const int W = (dct || pd.transform == TR_AR) ? n : half;
  const std::vector<double>& H = h.psf_pre;
  std::vector<double> q, tab;
  if (pd.transform == TR_AR) {
    // cos(pi m/(n-1)), m < 2(n-1); angle index k for the sine vectors, 0 for
    // the two linear ones (k = 0, n-1)
    const int per = 2 * (n - 1);
    tab.resize(per);
    for (int m = 0; m < per; ++m) tab[m] = std::cos(M_PI * (double)m / (double)(n - 1));
    q.assign((size_t)p * n, 0.0);
    for (int a = 0; a < p; ++a)
      for (int k2 = 0; k2 < n; ++k2) {
        const int kk = (k2 == n - 1) ? 0 : k2;
        double s = 0;
        for (int b = 0; b < p; ++b) {
          int m = (kk * (b - c)) % per; if (m < 0) m += per;
          s += H[a * p + b] * tab[m];
        }
        q[(size_t)a * n + k2] = s;
      }
  } else if (dct) {
    tab.resize(2 * n);
    for (int m = 0; m < 2 * n; ++m) tab[m] = std::cos(M_PI * (double)m / (double)n);
    q.assign((size_t)p * n, 0.0);
    for (int a = 0; a < p; ++a)
      for (int k2 = 0; k2 < n; ++k2) {
        double s = 0;
        for (int b = 0; b < p; ++b) {
          int m = (k2 * (b - c)) % (2 * n); if (m < 0) m += 2 * n;
          s += H[a * p + b] * tab[m];
        }
        q[(size_t)a * n + k2] = s;
      }
  } else {
    tab.resize(2 * n);
    for (int m = 0; m < n; ++m) {
      const double ang = 2.0 * M_PI * (double)m / (double)n;
      tab[2 * m] = std::cos(ang); tab[2 * m + 1] = -std::sin(ang);
    }
    q.assign((size_t)p * half * 2, 0.0);
    for (int a = 0; a < p; ++a)
      for (int k2 = 0; k2 < half; ++k2) {
        double re = 0, im = 0;
        for (int b = 0; b < p; ++b) {
          int m = (k2 * (b - c)) % n; if (m < 0) m += n;
          re += H[a * p + b] * tab[2 * m]; im += H[a * p + b] * tab[2 * m + 1];
        }
        q[2 * ((size_t)a * half + k2)] = re; q[2 * ((size_t)a * half + k2) + 1] = im;
      }
  }
  double *dq = nullptr, *dtab = nullptr;
  CK(cudaMalloc(&dq, q.size() * sizeof(double)));
  CK(cudaMalloc(&dtab, tab.size() * sizeof(double)));
  CK(cudaMemcpyAsync(dq, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  launch_spectrum_setup(pd.transform, n, p, half, pd.cb, dq, dtab, pd.lam, pd.w,
                        B->dtype == MLBA_F64 ? 1 : 0, B->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(B->stream));
  cudaFree(dq);
  cudaFree(dtab);
  (void)W;
  return MLBA_OK;
}

// ---- tile-shape autotuner of the framelet kernel ----------------------------
// The shape (warps per CTA, z prefetch distance) of the L <= 2 framelet
// launch is chosen per batch: forced by the options, read from the on-disk
// cache, or measured here (every candidate launched over the batch's own
// buffers, best of a few CUDA-event-timed launches).  All shapes give the same
// values, so the choice changes only the time.

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}

std::string tune_key(const mlba_batch* B) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) std::memset(&prop, 0, sizeof(prop));
  std::string name(prop.name);
  for (char& ch : name) if (ch == ' ' || ch == '\t') ch = '_';
  uint64_t h = 1469598103934665603ull;
  for (const HostProb& hp : B->hp) {
    const int v[5] = {hp.pd.n, hp.pd.nf, hp.pd.bc, hp.pd.use_adj, hp.pd.c};
    h = fnv1a(h, v, sizeof(v));
  }
  char buf[320];
  std::snprintf(buf, sizeof(buf), "frame3 %s sm%d%d dt%d zs%d L%d count%zu h%016llx",
                name.empty() ? "gpu" : name.c_str(), prop.major, prop.minor, B->dtype, B->z_store,
                B->levels, B->hp.size(), (unsigned long long)h);
  return std::string(buf);
}

std::string tune_cache_path() {
  if (const char* e = std::getenv("MLBA_TUNE_CACHE")) return std::string(e);
  if (const char* x = std::getenv("XDG_CACHE_HOME")) return std::string(x) + "/mlba_tune.txt";
  if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/mlba_tune.txt";
  return std::string();
}

bool tune_lookup(const std::string& key, int* shape, float* us) {
  const std::string path = tune_cache_path();
  if (path.empty()) return false;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    if (key != line) continue;
    int sh = -1;
    float t = 0.f;
    if (std::sscanf(tab + 1, "%d %f", &sh, &t) == 2 && sh >= 0 && sh < FRAME_SHAPES) {
      *shape = sh; *us = t; found = true;     // the last entry for a key wins
    }
  }
  std::fclose(f);
  return found;
}

void tune_store(const std::string& key, int shape, float us) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;                               // no writable cache: keep the choice in memory
  std::fprintf(f, "%s\t%d %.3f\n", key.c_str(), shape, us);
  std::fclose(f);
}

void launch_frame_any(mlba_batch* B, const int2* items, int count, int shape, cudaStream_t s) {
  if (B->dtype == MLBA_F64)
    launch_frame<double, double>(B->d_probs, B->d_states, items, count, nullptr, -1, SL_F, nullptr,
                                 nullptr, 0.0, B->levels, shape, s);
  else if (B->z_store == MLBA_BF16)
    launch_frame<float, __nv_bfloat16>(B->d_probs, B->d_states, items, count, nullptr, -1, SL_F,
                                       nullptr, nullptr, 0.0, B->levels, shape, s);
  else
    launch_frame<float, float>(B->d_probs, B->d_states, items, count, nullptr, -1, SL_F, nullptr,
                               nullptr, 0.0, B->levels, shape, s);
}

std::vector<int2> frame_items(const mlba_batch* B, int shape) {
  std::vector<int2> v;
  for (size_t i = 0; i < B->hp.size(); ++i) {
    const int nb = frame_tiles(B->hp[i].pd.nf, B->levels, shape);
    for (int k = 0; k < nb; ++k) v.push_back(make_int2((int)i, k));
  }
  return v;
}

// mean microseconds of one framelet launch of `shape` over the whole batch
int time_frame_shape(mlba_batch* B, int shape, float* us) {
  const std::vector<int2> items = frame_items(B, shape);
  int2* dev = nullptr;
  CK(cudaMalloc(&dev, items.size() * sizeof(int2)));
  if (cudaMemcpy(dev, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dev);
    return MLBA_E_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int warm = 2, reps = 6;
  for (int r = 0; r < warm; ++r) launch_frame_any(B, dev, (int)items.size(), shape, B->stream);
  cudaEventRecord(e0, B->stream);
  for (int r = 0; r < reps; ++r) launch_frame_any(B, dev, (int)items.size(), shape, B->stream);
  cudaEventRecord(e1, B->stream);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dev);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return MLBA_E_CUDA;
  *us = 1e3f * ms / reps;
  return MLBA_OK;
}

int choose_frame_shape(mlba_batch* B, const mlba_opts& o) {
  B->frame_shape = 0;
  B->frame_tuned = 0;
  const bool shaped = B->levels <= 2 && B->dtype != MLBA_F64;   // FP64: one shape
  if (!shaped) return MLBA_OK;
  if (o.frame_shape >= 0) {
    B->frame_shape = o.frame_shape;
    B->frame_tuned = 3;
    return MLBA_OK;
  }
  if (!o.autotune) return MLBA_OK;
  const std::string key = tune_key(B);
  int sh = 0;
  float us = 0.f;
  if (o.autotune == 1 && tune_lookup(key, &sh, &us)) {
    B->frame_shape = sh; B->frame_tuned = 2; B->frame_us = us;
    return MLBA_OK;
  }
  // the first step reads z^0 = 0 from z[0] and writes z[1]; the timed
  // launches read z[1] and write z[0], which the reset after create clears
  for (const HostProb& hp : B->hp)
    CK(cudaMemsetAsync(hp.pd.z[1], 0, (size_t)hp.pd.nbands * hp.pd.nf * hp.pd.nf * zsize(B->z_store),
                       B->stream));
  int best = 0;
  float tbest = 0.f;
  for (int k = 0; k < FRAME_SHAPES; ++k) {
    float t = 0.f;
    const int rc = time_frame_shape(B, k, &t);
    if (rc != MLBA_OK) return rc;
    if (k == 0 || t < tbest) { best = k; tbest = t; }
  }
  B->frame_shape = best; B->frame_tuned = 1; B->frame_us = tbest;
  tune_store(key, best, tbest);
  return MLBA_OK;
}

// ---- direct or FFT blur per problem (opts.blur_path 2) ----------------------
// A f of problem i alone by the direct stencil and by FFT convolution (the
// operator forms: no stop rule, states zeroed), best of a few CUDA-event-timed
// launches each; the problem keeps the faster.  Both compute A f: the choice
// changes the time (and the rounding), not the operator.
template <typename T>
int time_blur_paths(mlba_batch* B, int i, float* t_dir, float* t_fft) {
  const int count = (int)B->hp.size();
  const Prob& pd = B->hp[i].pd;
  const Prob& sf = B->fc[pd.fc_sh[0] - count].pd;
  const int fi = pd.fc_sh[0];
  std::vector<int2> st, pad, rows, cols, out;
  for (int k = 0; k < pd.nblk_blur; ++k) st.push_back(make_int2(i, k));
  for (int k = 0; k < sf.nblk_vec; ++k) pad.push_back(make_int2(fi, k));
  for (int k = 0; k < sf.nblk_rows; ++k) rows.push_back(make_int2(fi, k));
  for (int k = 0; k < sf.nblk_cols; ++k) cols.push_back(make_int2(fi, k));
  for (int k = 0; k < pd.nblk_vec; ++k) out.push_back(make_int2(i, k));
  ItemList L[5];
  const std::vector<int2>* v[5] = {&st, &pad, &rows, &cols, &out};
  for (int q = 0; q < 5; ++q)
    if (build_list(B, L[q], *v[q]) != MLBA_OK) return MLBA_E_CUDA;
  const Prob* P = B->d_probs;
  State* S = B->d_opstates;
  cudaStream_t s = B->stream;
  auto direct = [&] {
    launch_stencil<T>(ST_FWD_STORE, P, S, L[0].dev, L[0].count, SL_F, SL_AUX1, SL_AUX1, 0, B->smem_stencil, s);
  };
  auto fft = [&] {
    launch_fc_pad<T>(P, S, L[1].dev, L[1].count, 0, SL_F, s);
    launch_rows_fwd<T>(P, S, L[2].dev, L[2].count, SL_R, 0, B->smem_fft, s);
    launch_cols<T>(P, S, L[3].dev, L[3].count, COL_OP, 0, 1.0, W_TIKH, B->smem_fft, s);
    launch_rows_inv<T>(P, S, L[2].dev, L[2].count, SL_T, 0, B->smem_fft, s);
    launch_fc_out<T>(P, S, L[4].dev, L[4].count, FC_STORE_MODE, 0, SL_AUX1, s);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best[2] = {1e30f, 1e30f};
  for (int path = 0; path < 2; ++path)
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, s);
      if (path == 0) direct(); else fft();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return MLBA_E_CUDA; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) best[path] = std::min(best[path], ms);   // the first launch warms up
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  *t_dir = best[0];
  *t_fft = best[1];
  return MLBA_OK;
}

int choose_blur_paths(mlba_batch* B) {
  const int count = (int)B->hp.size();
  CK(cudaMemsetAsync(B->d_opstates, 0, count * sizeof(State), B->stream));
  for (int i = 0; i < count; ++i) {
    Prob& pd = B->hp[i].pd;
    if (pd.fc_sh[1] == 0) continue;               // no convolution entries
    float td = 0.f, tf = 0.f;
    const int rc = B->dtype == MLBA_F64 ? time_blur_paths<double>(B, i, &td, &tf)
                                        : time_blur_paths<float>(B, i, &td, &tf);
    if (rc != MLBA_OK) return rc;
    pd.fc = tf < td ? 1 : 0;
    CK(cudaMemcpy(&B->d_probs[i].fc, &pd.fc, sizeof(int), cudaMemcpyHostToDevice));
  }
  return MLBA_OK;
}

// ---- persistent schedule ----------------------------------------------------
// The stages of one step in the order of enqueue_step; stages in one group
// touch disjoint problems and share the grid barrier that ends the group.
int build_persist(mlba_batch* B) {
  const StepLists L = all_lists(B);
  std::vector<std::vector<PersistStage>> groups;
  auto st = [](int kind, const ItemList& l) {
    PersistStage p;
    p.kind = kind; p.count = l.count; p.items = l.dev; p.sync = 0; p.pad = 0;
    return p;
  };
  groups.push_back({st(PS_RESID, L.blur)});
  if (L.any_spec) {
    groups.push_back({st(PS_ROWS_FWD, L.rows_spec)});
    groups.push_back({st(PS_COLS_FUSED, L.cols_stat), st(PS_COLS_FWD, L.cols_ns)});
    if (L.any_ns) {
      for (int k = 1; k < ns_passes<float>(); ++k) groups.push_back({st(PS_SPEC, L.spec)});
      groups.push_back({st(PS_COLS_NSINV, L.cols_ns)});
    }
    groups.push_back({st(PS_ROWS_INV, L.rows_spec)});
  }
  groups.push_back({st(PS_CORR, L.corr), st(PS_REBLUR, L.reblur)});
  groups.push_back({st(PS_BALANCE, L.balance)});
  groups.push_back({st(PS_FRAME, L.frame)});
  std::vector<PersistStage> prog;
  for (const auto& g : groups) {
    const size_t first = prog.size();
    for (const PersistStage& p : g) if (p.count > 0) prog.push_back(p);
    if (prog.size() > first) prog.back().sync = 1;
  }
  B->nstages = (int)prog.size();
  CK(cudaMalloc(&B->d_stages, prog.size() * sizeof(PersistStage)));
  CK(cudaMemcpy(B->d_stages, prog.data(), prog.size() * sizeof(PersistStage), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&B->d_ctl, persist_ctl_bytes()));
  CK(cudaMemset(B->d_ctl, 0, persist_ctl_bytes()));
  // one stencil slot of the widest problem, the framelet slot, or a transform
  const int zsb = B->z_store == MLBA_BF16 ? 2 : 4;
  B->p_smem = persist_smem(4, zsb, B->levels, B->smem_stencil, B->smem_fft, &B->p_stencil_slot,
                           &B->p_frame_slot);
  const void* fn = persist_func(zsb, B->levels);
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->p_smem));
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, persist_threads(), B->p_smem));
  if (per_sm < 1) return MLBA_E_UNSUPPORTED;
  // no more CTAs than the largest stage has work for (two stencil items or
  // four framelet items per CTA): fewer arrivals at every grid barrier
  int need = 1;
  for (const PersistStage& p : prog) {
    const int per = (p.kind == PS_RESID || p.kind == PS_CORR || p.kind == PS_REBLUR) ? 2
                    : p.kind == PS_FRAME ? 4 : 1;
    need = std::max(need, (p.count + per - 1) / per);
  }
  B->p_grid = std::min(per_sm * sms, need);
  // the launch as a graph (one step; iterate(k) sets k in the instantiated copy)
  CK(persist_graph(zsb, B->levels, B->p_grid, B->p_smem, B->d_probs, B->d_states,
                   (int)B->hp.size(), B->d_stages, B->nstages, 1, B->d_ctl, B->p_wait_ns,
                   B->p_stencil_slot, B->p_frame_slot, &B->p_graph, &B->p_knode));
  CK(cudaGraphInstantiate(&B->p_exec, B->p_graph, 0));
  B->p_k = 1;
  B->persistent = true;
  return MLBA_OK;
}

int create_batch(const mlba_problem* probs, int count, const mlba_opts* opts_in, mlba_batch** out) {
  if (!probs || count <= 0 || !out) return MLBA_E_INVAL;
  mlba_opts o;
  if (opts_in) o = *opts_in; else mlba_opts_default(&o);
  if (o.dtype != MLBA_F32 && o.dtype != MLBA_F64) return MLBA_E_INVAL;
  if (o.dtype == MLBA_F64 && o.z_store != MLBA_F64) o.z_store = MLBA_F64;
  if (o.dtype == MLBA_F32 && o.z_store != MLBA_BF16) o.z_store = MLBA_F32;
  if (o.pcg_max < 1 || o.pcg_max > 50) return MLBA_E_INVAL;
  if (o.autotune < 0 || o.autotune > 2 || o.frame_shape < -1 || o.frame_shape >= FRAME_SHAPES)
    return MLBA_E_INVAL;
  if (o.blur_path < 0 || o.blur_path > 2) return MLBA_E_INVAL;
  if (o.formulation < 0 || o.formulation > 1) return MLBA_E_INVAL;
  if (o.persistent < 0 || o.persistent > 1 || !(o.wait_s >= 0.0) || o.wait_s > 1e3) return MLBA_E_INVAL;
  if (o.persistent) {
    if (o.dtype != MLBA_F32 || o.levels > 2 || o.blur_path != 0) return MLBA_E_UNSUPPORTED;
    o.frame_shape = 0;      // the persistent kernel's framelet body has the built-in shape
    o.two_group = 0;
  }
  mlba_batch* B = new (std::nothrow) mlba_batch();
  if (!B) return MLBA_E_NOMEM;
  B->dtype = o.dtype; B->z_store = o.z_store; B->levels = o.levels;
  B->hp.resize(count);
  for (int i = 0; i < count; ++i) {
    const int rc = setup_problem(probs[i], o, B->hp[i]);
    if (rc != MLBA_OK) { destroy_batch(B); return rc; }
    B->hp[i].pd.sidx = i;
    if (o.persistent && (B->hp[i].pd.precond == P_KRYLOV || B->hp[i].pd.transform == TR_AR)) {
      destroy_batch(B);
      return MLBA_E_UNSUPPORTED;
    }
  }
  // ---- FFT blur path: two convolution entries (forward, adjoint) for every
  // problem that may use it (Algorithm 2's PCG keeps the stencils; the
  // convolution size must fit one transform CTA)
  B->blur_path = o.blur_path;
  if (o.blur_path) {
    for (int i = 0; i < count; ++i) {
      HostProb& h = B->hp[i];
      if (h.pd.precond == P_KRYLOV) continue;
      HostProb sf, sa;
      if (!setup_conv_entry(h, i, 0, sf) || !setup_conv_entry(h, i, 1, sa)) continue;
      h.pd.fc_sh[0] = count + (int)B->fc.size();
      B->fc.push_back(sf);
      h.pd.fc_sh[1] = count + (int)B->fc.size();
      B->fc.push_back(sa);
      h.pd.fc = (o.blur_path == 1) ? 1 : 0;       // 2: measured below
    }
  }
  if (o.stream) { B->stream = (cudaStream_t)o.stream; }
  else {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      destroy_batch(B); return MLBA_E_CUDA;
    }
    B->own_stream = true;
  }
  const size_t ts = tsize(o.dtype), zs = zsize(o.z_store);
  // ---- arena layout
  size_t total = 0;
  std::vector<std::vector<size_t>> offs(count), szs(count);
  for (int i = 0; i < count; ++i) {
    Prob& pd = B->hp[i].pd;
    const size_t n2 = (size_t)pd.n * pd.n, nf2 = (size_t)pd.nf * pd.nf, ne2 = (size_t)pd.ne * pd.ne;
    const bool spec = pd.transform != TR_NONE;
    const bool kry = pd.precond == P_KRYLOV;
    const size_t nspec = spec ? spec_elems(pd) : 1;
    const size_t aux = std::max(nf2, ne2);
    std::vector<size_t> sz = {
        n2 * ts,                               // G
        nf2 * ts,                              // F
        n2 * ts,                               // R
        n2 * ts,                               // T
        ne2 * ts,                              // V
        n2 * ts,                               // U
        nspec * ts * (pd.transform == TR_DCT || pd.transform == TR_AR ? 1 : 2),   // S
        kry ? n2 * ts : ts, kry ? n2 * ts : ts, kry ? n2 * ts : ts, kry ? n2 * ts : ts,
        kry ? n2 * ts : ts,                    // PCG vectors
        aux * ts, aux * ts,                    // AUX0, AUX1
        (size_t)pd.nbands * nf2 * zs,          // z0
        (size_t)pd.nbands * nf2 * zs,          // z1
        nspec * ts * (pd.transform == TR_DCT || pd.transform == TR_AR ? 1 : 2),   // lam
        nspec * ts,                            // |lambda|^2 in T precision
        (pd.ns ? nspec : 1) * ts,              // 4-NS weighted power
        (pd.levels >= 3 ? (size_t)(pd.levels - 1) * nf2 : 1) * ts,   // low-pass chain (L >= 3)
        (pd.levels >= 3 ? (size_t)(pd.levels - 1) * nf2 : 1) * ts,   // synthesis partials
        pd.balanced ? (size_t)pd.nbands * nf2 * zs : zs,             // zeros (balanced z_in)
        spec ? (size_t)pd.nfft * 2 * ts : ts,  // tw
        spec ? (size_t)pd.n * 2 * ts : ts,     // dtw
        (size_t)pd.nruns * 16, 2 * (size_t)pd.nrw * ts,   // tap runs and weights (both orders)
        (size_t)pd.p * ts, (size_t)pd.p * ts,  // hy, hx
        std::max({3 * (size_t)pd.nblk_blur, 3 * (size_t)pd.nblk_vec, (size_t)SPEC_SUMS * std::max(pd.nblk_spec, pd.nblk_cols), (size_t)1}) * 8,  // partial
        (size_t)(pd.max_iter + 2) * 8, (size_t)(pd.max_iter + 2) * 8, (size_t)(pd.max_iter + 2) * 4};
    szs[i] = sz;
  }
  // f and z^0 of every problem come first, side by side, so that a reset
  // clears all of them with one memset of [arena, arena + zero_bytes); the
  // other buffers follow, problem by problem
  const size_t kF = SL_F, kZ0 = NSLOT;
  for (int i = 0; i < count; ++i) {
    offs[i].assign(szs[i].size(), 0);
    offs[i][kF] = total; total += al(szs[i][kF]);
    offs[i][kZ0] = total; total += al(szs[i][kZ0]);
  }
  B->zero_bytes = total;
  for (int i = 0; i < count; ++i)
    for (size_t k = 0; k < szs[i].size(); ++k)
      if (k != kF && k != kZ0) { offs[i][k] = total; total += al(szs[i][k]); }
  // convolution entries: X, Y, the spectrum work array, the two spectra, a
  // zero |lambda|^2 and the twiddles, shared by the pair of one problem (the
  // forward pass and the adjoint pass of a step never overlap)
  const size_t nfc = B->fc.size() / 2;
  std::vector<std::vector<size_t>> foffs(nfc);
  for (size_t k = 0; k < nfc; ++k) {
    const Prob& sf = B->fc[2 * k].pd;
    const size_t M2 = (size_t)sf.n * sf.n, nspec = spec_elems(sf);
    std::vector<size_t> sz = {M2 * ts, M2 * ts, nspec * 2 * ts, nspec * 2 * ts, nspec * 2 * ts,
                              nspec * ts, (size_t)sf.nfft * 2 * ts};
    foffs[k].resize(sz.size());
    for (size_t q = 0; q < sz.size(); ++q) { foffs[k][q] = total; total += al(sz[q]); }
  }
  B->arena_bytes = total;
  if (cudaMalloc(&B->arena, total) != cudaSuccess) {
    (void)cudaGetLastError();   // an allocation failure is not sticky: leave no stale error behind
    destroy_batch(B);
    return MLBA_E_NOMEM;
  }
  // ---- fill pointers and constant tables
  std::vector<unsigned char> host_init;   // staged constant data
  for (int i = 0; i < count; ++i) {
    HostProb& h = B->hp[i];
    Prob& pd = h.pd;
    const std::vector<size_t>& of = offs[i];
    unsigned char* base = B->arena;
    for (int s = 0; s < NSLOT; ++s) pd.buf[s] = base + of[s];
    int k = NSLOT;
    pd.z[0] = base + of[k++];
    pd.z[1] = base + of[k++];
    pd.lam = base + of[k++];
    pd.w = base + of[k++];
    pd.pw = base + of[k++];
    pd.lp = base + of[k++];
    pd.sy = base + of[k++];
    pd.z0 = base + of[k++];
    if (pd.balanced) CK(cudaMemset(pd.z0, 0, (size_t)pd.nbands * pd.nf * pd.nf * zs));
    else pd.z0 = nullptr;
    pd.tw = base + of[k++];
    pd.dtw = base + of[k++];
    pd.tap_runs = reinterpret_cast<int4*>(base + of[k++]);
    pd.tap_w = base + of[k++];
    pd.hy = base + of[k++];
    pd.hx = base + of[k++];
    pd.partial = reinterpret_cast<double*>(base + of[k++]);
    pd.hist_res = reinterpret_cast<double*>(base + of[k++]);
    pd.hist_alpha = reinterpret_cast<double*>(base + of[k++]);
    pd.hist_beta = reinterpret_cast<int*>(base + of[k++]);
    // tables
    CK(cudaMemcpy(pd.tap_runs, h.runs.data(), h.runs.size() * 4, cudaMemcpyHostToDevice));
    std::vector<unsigned char> tmp;
    auto upload = [&](void* dst, const std::vector<double>& v) -> int {
      tmp.assign(v.size() * ts, 0);
      if (ts == 8) put<double>(tmp.data(), 0, v); else put<float>(tmp.data(), 0, v);
      if (!v.empty()) CK(cudaMemcpy(dst, tmp.data(), tmp.size(), cudaMemcpyHostToDevice));
      return MLBA_OK;
    };
    if (upload(pd.tap_w, h.rw) != MLBA_OK) { destroy_batch(B); return MLBA_E_CUDA; }
    if (pd.sep) {
      if (upload(pd.hy, h.hy) != MLBA_OK || upload(pd.hx, h.hx) != MLBA_OK) {
        destroy_batch(B); return MLBA_E_CUDA;
      }
    }
    if (pd.transform != TR_NONE) {
      std::vector<double> tw(2 * (size_t)pd.nfft), dtw(2 * (size_t)pd.n);
      for (int m = 0; m < pd.nfft; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)pd.nfft;
        tw[2 * m] = std::cos(a); tw[2 * m + 1] = -std::sin(a);
      }
      for (int m = 0; m < pd.n; ++m) {
        const double b = M_PI * (double)m / (2.0 * (double)pd.n);
        dtw[2 * m] = std::cos(b); dtw[2 * m + 1] = -std::sin(b);
      }
      if (upload(pd.tw, tw) != MLBA_OK || upload(pd.dtw, dtw) != MLBA_OK) {
        destroy_batch(B); return MLBA_E_CUDA;
      }
      const int rc = build_spectrum(B, h);
      if (rc != MLBA_OK) { destroy_batch(B); return rc; }
    }
  }
  for (size_t k = 0; k < nfc; ++k) {
    unsigned char* base = B->arena;
    const std::vector<size_t>& of = foffs[k];
    for (int a = 0; a < 2; ++a) {
      Prob& pd = B->fc[2 * k + a].pd;
      pd.buf[SL_R] = base + of[0];
      pd.buf[SL_T] = base + of[1];
      pd.buf[SL_S] = base + of[2];
      pd.lam = base + of[3 + a];
      pd.w = base + of[5];
      pd.tw = pd.dtw = base + of[6];
    }
    const Prob& sf = B->fc[2 * k].pd;
    std::vector<double> tw(2 * (size_t)sf.nfft);
    for (int m = 0; m < sf.nfft; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)sf.nfft;
      tw[2 * m] = std::cos(a); tw[2 * m + 1] = -std::sin(a);
    }
    std::vector<unsigned char> tmp(tw.size() * ts);
    if (ts == 8) put<double>(tmp.data(), 0, tw); else put<float>(tmp.data(), 0, tw);
    if (cudaMemcpy(sf.tw, tmp.data(), tmp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      destroy_batch(B); return MLBA_E_CUDA;
    }
    for (int a = 0; a < 2; ++a) {
      const int rc = build_spectrum(B, B->fc[2 * k + a]);
      if (rc != MLBA_OK) { destroy_batch(B); return rc; }
    }
    // |lambda|^2 = 0: the column pass's weight is then conj(lambda) / M^2
    if (cudaMemset(sf.w, 0, spec_elems(sf) * ts) != cudaSuccess) { destroy_batch(B); return MLBA_E_CUDA; }
  }
  // ---- device tables (problems, then the convolution entries)
  const int ntab = count + (int)B->fc.size();
  std::vector<Prob> probs_h(ntab);
  std::vector<State> st_h(count);
  for (int i = 0; i < count; ++i) { probs_h[i] = B->hp[i].pd; st_h[i] = initial_state(probs_h[i]); }
  for (size_t k = 0; k < B->fc.size(); ++k) probs_h[count + k] = B->fc[k].pd;
  if (cudaMalloc(&B->d_probs, ntab * sizeof(Prob)) != cudaSuccess ||
      cudaMalloc(&B->d_states, count * sizeof(State)) != cudaSuccess ||
      cudaMalloc(&B->d_opstates, count * sizeof(State)) != cudaSuccess) {
    (void)cudaGetLastError();
    destroy_batch(B); return MLBA_E_NOMEM;
  }
  CK(cudaMemcpy(B->d_probs, probs_h.data(), ntab * sizeof(Prob), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B->d_states, st_h.data(), count * sizeof(State), cudaMemcpyHostToDevice));
  // ---- shared memory of the stencil and transform launches
  {
    size_t smem_st = 0, smem_fft = 0;
    for (int i = 0; i < count; ++i) {
      const Prob& pd = B->hp[i].pd;
      // stencil: weights (padded to 16 bytes), runs, input tile, row-pass tile
      const size_t RY = 32 + pd.p - 1, RX = 64 + pd.p - 1;
      const size_t ce = 16 / ts;                  // input-tile pitch as in k_stencil.cu (st_pitch)
      const size_t RP = (RX + 2 * (ce - 1)) / ce * ce;
      const size_t nw = pd.sep ? 2 * pd.p : pd.nrw;
      // (a second row-pass tile only for rank-one PSFs with 8 RY > 4 x 128, see k_stencil.cu)
      const size_t st_b = (((nw + 3) & ~(size_t)3) + RY * RP + (pd.sep && 8 * RY > 4 * 128 ? RY * 66 : 0)) * ts +
                          (pd.sep ? 0 : (size_t)pd.nruns * 16);
      smem_st = std::max(smem_st, st_b);
      if (pd.transform != TR_NONE) {
        // (antireflective columns also keep two weighted end values per transform)
        const size_t fb = (size_t)std::max(pd.row_g, pd.col_g) * (fft_pad(pd.nfft) + 1) * 2 * ts +
                          (pd.transform == TR_AR ? (size_t)pd.col_g * 4 * ts : 0);
        smem_fft = std::max(smem_fft, fb);
      }
    }
    for (const HostProb& h : B->fc) {
      const Prob& pd = h.pd;
      smem_fft = std::max(smem_fft, (size_t)std::max(pd.row_g, pd.col_g) * (fft_pad(pd.nfft) + 1) * 2 * ts);
    }
    B->smem_stencil = std::max<size_t>(smem_st, 16);
    B->smem_fft = std::max<size_t>(smem_fft, 16);
  }
  if (set_smem_attrs(B) != MLBA_OK) { destroy_batch(B); return MLBA_E_CUDA; }
  // ---- FFT or direct blur per problem (blur_path 2: the faster, measured)
  if (o.blur_path == 2) {
    const int rc = choose_blur_paths(B);
    if (rc != MLBA_OK) { destroy_batch(B); return rc; }
  }
  // ---- item lists
  std::vector<int2> blur, corr, reblur, corr_kry, blur_kry, rows_spec, cols_stat, cols_ns, spec,
      rows_kry, cols_kry, vec_kry, vec_kry_bc, corr_all, rows_all, cols_all, spec_all, vec_all,
      ar_rows, ar_cols;
  StepItems fcv;
  for (int i = 0; i < count; ++i) {
    const Prob& pd = B->hp[i].pd;
    auto add = [&](std::vector<int2>& L, int nblk) { for (int k = 0; k < nblk; ++k) L.push_back(make_int2(i, k)); };
    if (!pd.fc) add(blur, pd.nblk_blur);
    add(corr_all, pd.nblk_corr);
    add(vec_all, pd.nblk_vec);
    if (pd.use_adj && !pd.fc) {
      if (pd.bc == BC_AR) add(reblur, pd.nblk_blur);
      else add(corr, pd.nblk_corr);
    }
    if (pd.balanced) add(fcv.balance, vec_blocks((size_t)pd.nf * pd.nf));
    const bool specp = pd.transform != TR_NONE;
    if (specp) { add(rows_all, pd.nblk_rows); add(cols_all, pd.nblk_cols); add(spec_all, pd.nblk_spec); }
    if (pd.precond == P_KRYLOV) {
      add(corr_kry, pd.nblk_corr); add(blur_kry, pd.nblk_blur); add(rows_kry, pd.nblk_rows);
      add(cols_kry, pd.nblk_cols); add(vec_kry, pd.nblk_vec);
      if (pd.bc != BC_RECT) add(vec_kry_bc, pd.nblk_vec);
      B->any_krylov = 1;
    } else if (pd.transform == TR_AR) {
      add(ar_rows, pd.nblk_rows); add(ar_cols, pd.nblk_cols);
      B->any_ar = 1;
    } else if (specp) {
      add(rows_spec, pd.nblk_rows);
      B->any_spec = 1;
      if (pd.ns) { add(cols_ns, pd.nblk_cols); add(spec, pd.nblk_spec); B->any_ns = 1; }
      else { add(cols_stat, pd.nblk_cols); B->any_stat = 1; }
    }
    if (pd.fc)
      collect_fc(pd, i, B->fc[pd.fc_sh[0] - count].pd, B->fc[pd.fc_sh[1] - count].pd, fcv);
  }
  int rc = MLBA_OK;
  {
    StepLists fl;
    rc |= build_fc_lists(B, fl, fcv);
    B->fc_pad_f = fl.fc_pad_f; B->fc_rows_f = fl.fc_rows_f; B->fc_cols_f = fl.fc_cols_f;
    B->fc_out_r = fl.fc_out_r; B->fc_pad_a = fl.fc_pad_a; B->fc_rows_a = fl.fc_rows_a;
    B->fc_cols_a = fl.fc_cols_a; B->fc_out_v = fl.fc_out_v; B->fc_out_u = fl.fc_out_u;
    rc |= build_list(B, B->balance, fcv.balance);
  }
  rc |= build_list(B, B->blur, blur); rc |= build_list(B, B->corr, corr);
  rc |= build_list(B, B->reblur, reblur);
  rc |= build_list(B, B->corr_kry, corr_kry); rc |= build_list(B, B->blur_kry, blur_kry);
  rc |= build_list(B, B->rows_spec, rows_spec); rc |= build_list(B, B->cols_stat, cols_stat);
  rc |= build_list(B, B->cols_ns, cols_ns); rc |= build_list(B, B->spec, spec);
  rc |= build_list(B, B->rows_kry, rows_kry); rc |= build_list(B, B->cols_kry, cols_kry);
  rc |= build_list(B, B->vec_kry, vec_kry); rc |= build_list(B, B->vec_kry_bc, vec_kry_bc);
  rc |= build_list(B, B->corr_all, corr_all);
  rc |= build_list(B, B->rows_all, rows_all); rc |= build_list(B, B->cols_all, cols_all);
  rc |= build_list(B, B->spec_all, spec_all); rc |= build_list(B, B->vec_all, vec_all);
  rc |= build_list(B, B->ar_rows, ar_rows); rc |= build_list(B, B->ar_cols, ar_cols);
  if (rc != MLBA_OK) { destroy_batch(B); return MLBA_E_CUDA; }
  // ---- framelet tile shape, then the framelet list in that shape
  {
    const int trc = choose_frame_shape(B, o);
    if (trc != MLBA_OK) { destroy_batch(B); return trc; }
    std::vector<int2> fs[FRAME_SECTIONS];
    for (int i = 0; i < count; ++i) add_frame_items(B->hp[i].pd, i, B->levels, B->frame_shape, fs);
    if (build_frame_list(B, B->frame, fs, B->levels) != MLBA_OK) { destroy_batch(B); return MLBA_E_CUDA; }
  }
  // ---- capture one step (branch streams first: a capture forks into them)
  for (int q = 0; q < 2; ++q) {
    if (cudaStreamCreateWithFlags(&B->br[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_bf[q], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_bj[q], cudaEventDisableTiming) != cudaSuccess) {
      destroy_batch(B); return MLBA_E_CUDA;
    }
  }
  if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    destroy_batch(B); return MLBA_E_CUDA;
  }
  enqueue_dispatch(B, all_lists(B), PART_ALL, B->stream);
  if (cudaStreamEndCapture(B->stream, &B->graph) != cudaSuccess ||
      cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess) {
    destroy_batch(B); return MLBA_E_CUDA;
  }
  if (o.two_group && build_split(B) != MLBA_OK) { destroy_batch(B); return MLBA_E_CUDA; }
  if (o.persistent) {
    B->p_wait_ns = (unsigned long long)(o.wait_s * 1e9);
    const int prc = build_persist(B);
    if (prc != MLBA_OK) { destroy_batch(B); return prc; }
  }
  *out = B;
  return MLBA_OK;
}

int reset_batch(mlba_batch* B) {
  std::vector<State> st_h(B->hp.size());
  // f and z^0 of every problem: one region at the start of the arena
  CK(cudaMemsetAsync(B->arena, 0, B->zero_bytes, B->stream));
  for (size_t i = 0; i < B->hp.size(); ++i) st_h[i] = initial_state(B->hp[i].pd);
  CK(cudaMemcpyAsync(B->d_states, st_h.data(), st_h.size() * sizeof(State), cudaMemcpyHostToDevice,
                     B->stream));
  CK(cudaStreamSynchronize(B->stream));
  return MLBA_OK;
}

int set_g(mlba_batch* B, int i, const void* g, int on_device, double delta) {
  HostProb& h = B->hp[i];
  const size_t bytes = (size_t)h.pd.n * h.pd.n * tsize(B->dtype);
  if (!g) return MLBA_E_INVAL;
  CK(cudaMemcpyAsync(h.pd.buf[SL_G], g, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     B->stream));
  if (delta != h.pd.delta) {
    h.pd.delta = delta;
    CK(cudaMemcpyAsync(&B->d_probs[i].delta, &h.pd.delta, sizeof(double), cudaMemcpyHostToDevice, B->stream));
  }
  CK(cudaStreamSynchronize(B->stream));
  return MLBA_OK;
}

int copy_out(mlba_batch* B, void* dst, const void* src, size_t bytes, int on_device) {
  if (!dst) return MLBA_E_INVAL;
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, B->stream));
  if (!on_device) CK(cudaStreamSynchronize(B->stream));
  return MLBA_OK;
}

int copy_in(mlba_batch* B, void* dst, const void* src, size_t bytes, int on_device) {
  if (!src) return MLBA_E_INVAL;
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, B->stream));
  return MLBA_OK;
}

int stats_of(mlba_batch* B, int i, mlba_stats* s) {
  if (!s || i < 0 || i >= (int)B->hp.size()) return MLBA_E_INVAL;
  State st;
  CK(cudaMemcpyAsync(&st, &B->d_states[i], sizeof(State), cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  s->iter = st.iter;
  s->stopped = st.stopped;
  s->stop_iter = st.stop_iter;
  s->status = st.status;
  s->resnorm = st.resnorm;
  s->alpha_n = st.alpha_n;
  s->beta_n = st.beta_last;
  s->nres = st.nres;
  return MLBA_OK;
}

int reset_opstates(mlba_batch* B) {
  CK(cudaMemsetAsync(B->d_opstates, 0, B->hp.size() * sizeof(State), B->stream));
  return MLBA_OK;
}

}  // namespace

// ============================================================================
// C ABI
extern "C" {

void mlba_opts_default(mlba_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mu = 10.0 / 255.0;
  o->alpha = 0.05;
  o->gamma = 1.0 + 1e-15;
  o->q = 0.5;
  o->rho = 1e-4;
  o->pcg_tol = 1e-3;
  o->levels = 1;
  o->max_iter = 200;
  o->pcg_max = 5;
  o->two_group = 1;
  o->dtype = MLBA_F32;
  o->z_store = MLBA_F32;
  o->transform = MLBA_TR_AUTO;
  o->stop = 1;
  o->rect_ns_hybrid = 0;
  o->stream = nullptr;
  o->autotune = 0;
  o->frame_shape = -1;
  o->blur_path = 0;
  o->formulation = 0;
  o->persistent = 0;
  o->wait_s = 1.0;
}

const char* mlba_strerror(int s) {
  switch (s) {
    case MLBA_OK: return "ok";
    case MLBA_E_INVAL: return "invalid argument";
    case MLBA_E_NOMEM: return "out of memory";
    case MLBA_E_CUDA: return "CUDA runtime error";
    case MLBA_E_TIMEOUT: return "device wait timed out";
    case MLBA_E_DIVERGED: return "residual norm not finite (diverged)";
    case MLBA_E_STATE: return "call out of order";
    case MLBA_E_UNSUPPORTED: return "unsupported size";
    default: return "unknown status";
  }
}

int mlba_batch_create(const mlba_problem* probs, int count, const mlba_opts* opts, mlba_batch** out) {
  if (!out) return MLBA_E_INVAL;
  *out = nullptr;
  mlba_batch* B = nullptr;
  int rc = create_batch(probs, count, opts, &B);
  if (rc != MLBA_OK) return rc;
  for (int i = 0; i < count; ++i) {
    if (probs[i].g) {
      rc = set_g(B, i, probs[i].g, probs[i].g_on_device, probs[i].delta);
      if (rc != MLBA_OK) { destroy_batch(B); return rc; }
    }
  }
  rc = reset_batch(B);
  if (rc != MLBA_OK) { destroy_batch(B); return rc; }
  B->has_data = true;
  for (int i = 0; i < count; ++i) if (!probs[i].g) B->has_data = false;
  *out = B;
  return MLBA_OK;
}

int mlba_batch_iterate(mlba_batch* B, int k) {
  if (!B || k < 0) return MLBA_E_INVAL;
  if (!B->has_data) return MLBA_E_STATE;
  if (k == 0) return MLBA_OK;
  if (B->persistent) {
    // one graph launch: the barrier words cleared, then the k steps in one
    // cooperative kernel
    if (k != B->p_k) {
      CK(persist_graph_set_k(B->p_exec, B->p_knode, B->z_store == MLBA_BF16 ? 2 : 4, B->levels,
                             B->p_grid, B->p_smem, B->d_probs, B->d_states, (int)B->hp.size(),
                             B->d_stages, B->nstages, k, B->d_ctl, B->p_wait_ns,
                             B->p_stencil_slot, B->p_frame_slot));
      B->p_k = k;
    }
    CK(cudaGraphLaunch(B->p_exec, B->stream));
    return MLBA_OK;
  }
  if (B->split) {
    CK(cudaGraphLaunch(B->x_head, B->stream));
    for (int i = 1; i < k; ++i) CK(cudaGraphLaunch(B->x_body, B->stream));
    CK(cudaGraphLaunch(B->x_tail, B->stream));
    return MLBA_OK;
  }
  for (int i = 0; i < k; ++i) CK(cudaGraphLaunch(B->exec, B->stream));
  return MLBA_OK;
}

int mlba_batch_active(mlba_batch* B, int* n_active) {
  if (!B || !n_active) return MLBA_E_INVAL;
  std::vector<State> st(B->hp.size());
  CK(cudaMemcpyAsync(st.data(), B->d_states, st.size() * sizeof(State), cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  int a = 0;
  for (const State& s : st) a += s.stopped ? 0 : 1;
  *n_active = a;
  return MLBA_OK;
}

int mlba_batch_result(mlba_batch* B, int i, void* f_out, int on_device) {
  if (!B || i < 0 || i >= (int)B->hp.size()) return MLBA_E_INVAL;
  const Prob& pd = B->hp[i].pd;
  return copy_out(B, f_out, pd.buf[SL_F], (size_t)pd.nf * pd.nf * tsize(B->dtype), on_device);
}

int mlba_batch_stats(mlba_batch* B, int i, mlba_stats* st) {
  if (!B) return MLBA_E_INVAL;
  return stats_of(B, i, st);
}

int mlba_batch_reset(mlba_batch* B) {
  if (!B) return MLBA_E_INVAL;
  return reset_batch(B);
}

int mlba_batch_set_data(mlba_batch* B, int i, const void* g, int on_device, double delta) {
  if (!B || i < 0 || i >= (int)B->hp.size() || !g || !(delta >= 0.0)) return MLBA_E_INVAL;
  if (B->hp[i].pd.ns && !(delta > 0.0)) return MLBA_E_INVAL;
  return set_g(B, i, g, on_device, delta);
}

int mlba_batch_set_data_all(mlba_batch* B, const void* const* g, int on_device, const double* delta) {
  if (!B || !g || !delta) return MLBA_E_INVAL;
  const int count = (int)B->hp.size();
  for (int i = 0; i < count; ++i) {
    if (!g[i] || !(delta[i] >= 0.0)) return MLBA_E_INVAL;
    if (B->hp[i].pd.ns && !(delta[i] > 0.0)) return MLBA_E_INVAL;
  }
  for (int i = 0; i < count; ++i) {
    HostProb& h = B->hp[i];
    const size_t bytes = (size_t)h.pd.n * h.pd.n * tsize(B->dtype);
    CK(cudaMemcpyAsync(h.pd.buf[SL_G], g[i], bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, B->stream));
    if (delta[i] != h.pd.delta) {
      h.pd.delta = delta[i];
      CK(cudaMemcpyAsync(&B->d_probs[i].delta, &h.pd.delta, sizeof(double), cudaMemcpyHostToDevice,
                         B->stream));
    }
  }
  CK(cudaStreamSynchronize(B->stream));
  B->has_data = true;
  return MLBA_OK;
}

int mlba_batch_result_all(mlba_batch* B, void* const* f_out, int on_device) {
  if (!B || !f_out) return MLBA_E_INVAL;
  const int count = (int)B->hp.size();
  for (int i = 0; i < count; ++i)
    if (!f_out[i]) return MLBA_E_INVAL;
  for (int i = 0; i < count; ++i) {
    const Prob& pd = B->hp[i].pd;
    CK(cudaMemcpyAsync(f_out[i], pd.buf[SL_F], (size_t)pd.nf * pd.nf * tsize(B->dtype),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, B->stream));
  }
  if (!on_device) CK(cudaStreamSynchronize(B->stream));
  return MLBA_OK;
}

int mlba_batch_profile(mlba_batch* B, int stage, int reps, float* ms) {
  if (!B || !ms || reps < 1 || stage < 0 || stage > 4) return MLBA_E_INVAL;
  if (!B->has_data) return MLBA_E_STATE;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const Prob* P = B->d_probs;
  State* S = B->d_states;
  cudaStream_t s = B->stream;
  CK(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) {
    if (stage == 0) {
      CK(cudaGraphLaunch(B->exec, s));
    } else if (B->dtype == MLBA_F64) {
      if (stage == 1) launch_stencil<double>(ST_FWD_RESID, P, S, B->blur.dev, B->blur.count, SL_F, SL_R, SL_G, 0, B->smem_stencil, s);
      if (stage == 2) {
        launch_rows_fwd<double>(P, S, B->rows_spec.dev, B->rows_spec.count, SL_R, 0, B->smem_fft, s);
        launch_cols<double>(P, S, B->cols_stat.dev, B->cols_stat.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, s);
        launch_cols<double>(P, S, B->cols_ns.dev, B->cols_ns.count, COL_FWD, 0, 0.0, 0, B->smem_fft, s);
        launch_cols<double>(P, S, B->cols_ns.dev, B->cols_ns.count, COL_NS_INV, 0, 0.0, 0, B->smem_fft, s);
        launch_rows_inv<double>(P, S, B->rows_spec.dev, B->rows_spec.count, SL_T, 0, B->smem_fft, s);
        launch_ar_rows<double>(P, S, B->ar_rows.dev, B->ar_rows.count, SL_R, 0, 0, B->smem_fft, s);
        launch_ar_cols<double>(P, S, B->ar_cols.dev, B->ar_cols.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, s);
        launch_ar_rows<double>(P, S, B->ar_rows.dev, B->ar_rows.count, SL_T, 1, 0, B->smem_fft, s);
      }
      if (stage == 3) {
        launch_stencil<double>(ST_CORR, P, S, B->corr.dev, B->corr.count, -1, SL_V, SL_V, 0, B->smem_stencil, s);
        launch_stencil<double>(ST_REBLUR, P, S, B->reblur.dev, B->reblur.count, -1, -1, SL_U, 0, B->smem_stencil, s);
      }
      if (stage == 4) launch_frame<double, double>(P, S, B->frame.dev, B->frame.count, B->frame.sec, -1, SL_F, nullptr, nullptr, 0.0, B->levels, B->frame_shape, s);
    } else {
      if (stage == 1) launch_stencil<float>(ST_FWD_RESID, P, S, B->blur.dev, B->blur.count, SL_F, SL_R, SL_G, 0, B->smem_stencil, s);
      if (stage == 2) {
        launch_rows_fwd<float>(P, S, B->rows_spec.dev, B->rows_spec.count, SL_R, 0, B->smem_fft, s);
        launch_cols<float>(P, S, B->cols_stat.dev, B->cols_stat.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, s);
        launch_cols<float>(P, S, B->cols_ns.dev, B->cols_ns.count, COL_FWD, 0, 0.0, 0, B->smem_fft, s);
        launch_cols<float>(P, S, B->cols_ns.dev, B->cols_ns.count, COL_NS_INV, 0, 0.0, 0, B->smem_fft, s);
        launch_rows_inv<float>(P, S, B->rows_spec.dev, B->rows_spec.count, SL_T, 0, B->smem_fft, s);
        launch_ar_rows<float>(P, S, B->ar_rows.dev, B->ar_rows.count, SL_R, 0, 0, B->smem_fft, s);
        launch_ar_cols<float>(P, S, B->ar_cols.dev, B->ar_cols.count, COL_FUSED, 0, 0.0, 0, B->smem_fft, s);
        launch_ar_rows<float>(P, S, B->ar_rows.dev, B->ar_rows.count, SL_T, 1, 0, B->smem_fft, s);
      }
      if (stage == 3) {
        launch_stencil<float>(ST_CORR, P, S, B->corr.dev, B->corr.count, -1, SL_V, SL_V, 0, B->smem_stencil, s);
        launch_stencil<float>(ST_REBLUR, P, S, B->reblur.dev, B->reblur.count, -1, -1, SL_U, 0, B->smem_stencil, s);
      }
      if (stage == 4) {
        if (B->z_store == MLBA_BF16)
          launch_frame<float, __nv_bfloat16>(P, S, B->frame.dev, B->frame.count, B->frame.sec, -1, SL_F, nullptr, nullptr, 0.0, B->levels, B->frame_shape, s);
        else
          launch_frame<float, float>(P, S, B->frame.dev, B->frame.count, B->frame.sec, -1, SL_F, nullptr, nullptr, 0.0, B->levels, B->frame_shape, s);
      }
    }
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / (float)reps;
  return MLBA_OK;
}

int mlba_batch_tiles(mlba_batch* B, int* frame_shape, int* tile_x, int* tile_y, int* prefetch,
                     int* how, float* us);

int mlba_batch_graph_kernels(mlba_batch* B, int* n) {
  if (!B || !n || !B->graph) return MLBA_E_INVAL;
  // kernels of one step: the body graph of the two-group schedule holds one
  // step of each group
  cudaGraph_t g = B->split ? B->g_body : B->graph;
  size_t cnt = 0;
  CK(cudaGraphGetNodes(g, nullptr, &cnt));
  std::vector<cudaGraphNode_t> nodes(cnt);
  CK(cudaGraphGetNodes(g, nodes.data(), &cnt));
  int k = 0;
  for (size_t i = 0; i < cnt; ++i) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *n = k;
  return MLBA_OK;
}

void mlba_batch_destroy(mlba_batch* B) { destroy_batch(B); }

int mlba_batch_tiles(mlba_batch* B, int* frame_shape, int* tile_x, int* tile_y, int* prefetch,
                     int* how, float* us) {
  if (!B) return MLBA_E_INVAL;
  int tx = 0, ty = 0, pf = 0;
  if (B->levels <= 2) frame_shape_of(B, &tx, &ty, &pf);
  if (frame_shape) *frame_shape = B->frame_shape;
  if (tile_x) *tile_x = tx;
  if (tile_y) *tile_y = ty;
  if (prefetch) *prefetch = pf;
  if (how) *how = B->frame_tuned;
  if (us) *us = B->frame_us;
  return MLBA_OK;
}

// ---- single problem ---------------------------------------------------------
int mlba_create(const double* psf, int p, int n, int bc, int precond, const mlba_opts* opts,
                mlba_ctx** out) {
  if (!out) return MLBA_E_INVAL;
  *out = nullptr;
  mlba_opts o;
  if (opts) o = *opts; else mlba_opts_default(&o);
  mlba_problem pr;
  std::memset(&pr, 0, sizeof(pr));
  pr.psf = psf; pr.p = p; pr.n = n; pr.bc = bc; pr.precond = precond; pr.transform = o.transform;
  pr.max_iter = o.max_iter; pr.mu = o.mu; pr.alpha = o.alpha;
  pr.delta = precond == MLBA_P_TIKH_NS ? 1.0 : 0.0;   // placeholder until set_data
  pr.g = nullptr;
  mlba_batch* B = nullptr;
  int rc = create_batch(&pr, 1, &o, &B);
  if (rc != MLBA_OK) return rc;
  mlba_ctx* c = new (std::nothrow) mlba_ctx();
  if (!c) { destroy_batch(B); return MLBA_E_NOMEM; }
  c->b = B;
  *out = c;
  return MLBA_OK;
}

int mlba_batch_blur_fft(mlba_batch* B, int i, int* uses_fft, int* size) {
  if (!B || i < 0 || i >= (int)B->hp.size()) return MLBA_E_INVAL;
  const Prob& pd = B->hp[i].pd;
  if (uses_fft) *uses_fft = pd.fc;
  if (size) *size = pd.fc ? B->fc[pd.fc_sh[0] - (int)B->hp.size()].pd.n : 0;
  return MLBA_OK;
}

int mlba_tiles(mlba_ctx* c, int* frame_shape, int* tile_x, int* tile_y, int* prefetch, int* how,
               float* us) {
  if (!c) return MLBA_E_INVAL;
  return mlba_batch_tiles(c->b, frame_shape, tile_x, tile_y, prefetch, how, us);
}

int mlba_set_data(mlba_ctx* c, const void* g, int on_device, double delta) {
  if (!c || !g || !(delta >= 0.0)) return MLBA_E_INVAL;
  if (c->b->hp[0].pd.ns && !(delta > 0.0)) return MLBA_E_INVAL;
  int rc = set_g(c->b, 0, g, on_device, delta);
  if (rc != MLBA_OK) return rc;
  rc = reset_batch(c->b);
  if (rc != MLBA_OK) return rc;
  c->b->has_data = true;
  return MLBA_OK;
}

int mlba_iterate(mlba_ctx* c, int k) {
  if (!c) return MLBA_E_INVAL;
  return mlba_batch_iterate(c->b, k);
}

int mlba_result(mlba_ctx* c, void* f_out, int on_device) {
  if (!c) return MLBA_E_INVAL;
  return mlba_batch_result(c->b, 0, f_out, on_device);
}

int mlba_stats_get(mlba_ctx* c, mlba_stats* st) {
  if (!c) return MLBA_E_INVAL;
  return stats_of(c->b, 0, st);
}

int mlba_history(mlba_ctx* c, double* res, double* alpha, int* beta, int cap) {
  if (!c || cap < 0) return MLBA_E_INVAL;
  mlba_stats s;
  int rc = stats_of(c->b, 0, &s);
  if (rc != MLBA_OK) return rc;
  const Prob& pd = c->b->hp[0].pd;
  const int nres = std::min(s.nres, std::min(cap, pd.max_iter + 2));
  const int nit = std::min(s.iter, std::min(cap, pd.max_iter + 2));
  if (res && nres > 0) CK(cudaMemcpy(res, pd.hist_res, nres * sizeof(double), cudaMemcpyDeviceToHost));
  if (alpha && nit > 0) CK(cudaMemcpy(alpha, pd.hist_alpha, nit * sizeof(double), cudaMemcpyDeviceToHost));
  if (beta && nit > 0) CK(cudaMemcpy(beta, pd.hist_beta, nit * sizeof(int), cudaMemcpyDeviceToHost));
  return nres;
}

int mlba_get_z(mlba_ctx* c, void* z_out, int on_device) {
  if (!c) return MLBA_E_INVAL;
  mlba_stats s;
  int rc = stats_of(c->b, 0, &s);
  if (rc != MLBA_OK) return rc;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  const size_t es = zsize(B->z_store), plane = (size_t)pd.nf * pd.nf;
  const size_t zbytes = (size_t)pd.nbands * plane * es;
  if (!z_grouped(pd.levels)) return copy_out(B, z_out, pd.z[s.iter & 1], zbytes, on_device);
  if (!z_out) return MLBA_E_INVAL;
  // the library keeps z in its internal order (z_index); the caller gets band-major planes
  if (on_device) {
    launch_z_layout(z_out, pd.z[s.iter & 1], pd.levels, pd.nf, (int)es, 0, B->stream);
    CK(cudaGetLastError());
    return MLBA_OK;
  }
  std::vector<unsigned char> raw(zbytes);
  CK(cudaMemcpyAsync(raw.data(), pd.z[s.iter & 1], zbytes, cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  unsigned char* out = static_cast<unsigned char*>(z_out);
  for (int b = 0; b < pd.nbands; ++b)
    for (size_t q = 0; q < plane; ++q)
      std::memcpy(out + ((size_t)b * plane + q) * es,
                  raw.data() + z_index(b, (int)(q / pd.nf), (int)(q % pd.nf), pd.levels, pd.nf) * es,
                  es);
  return MLBA_OK;
}

}  // extern "C"

namespace {

// layout of the state blob of mlba_get_state / mlba_set_state
struct StateHeader {
  uint32_t magic, version;
  int32_t n, nf, p, bc, nbands, dtype, z_store, max_iter;
  int32_t precond, transform, stop, pcg_max, formulation;
  int32_t iter, stopped, stop_iter, status, nres, beta_last;
  double mu, alpha, gamma, delta, q, rho, pcg_tol;   // the iteration's parameters
  double resnorm, alpha_n, nb, qn;
};
constexpr uint32_t STATE_MAGIC = 0x4d4c4253u;   // "MLBS"
constexpr uint32_t STATE_VERSION = 3;

// the parameters that decide how the iteration continues, as the header keeps them
void header_params(const Prob& pd, StateHeader& h) {
  h.precond = pd.precond; h.transform = pd.transform; h.stop = pd.stop; h.pcg_max = pd.pcg_max;
  h.formulation = pd.balanced;
  h.mu = pd.mu; h.alpha = pd.alpha; h.gamma = pd.gamma; h.delta = pd.delta;
  h.q = pd.q; h.rho = pd.rho; h.pcg_tol = pd.pcg_tol;
}
bool same_params(const StateHeader& a, const StateHeader& b) {
  return a.precond == b.precond && a.transform == b.transform && a.stop == b.stop &&
         a.formulation == b.formulation &&
         a.pcg_max == b.pcg_max && a.mu == b.mu && a.alpha == b.alpha && a.gamma == b.gamma &&
         a.delta == b.delta && a.q == b.q && a.rho == b.rho && a.pcg_tol == b.pcg_tol;
}

struct StateLayout {
  size_t hist, f, z, total;
};
StateLayout state_layout(const mlba_batch* B) {
  const Prob& pd = B->hp[0].pd;
  const size_t cap = (size_t)pd.max_iter + 2;
  const size_t plane = (size_t)pd.nf * pd.nf;
  StateLayout L;
  L.hist = sizeof(StateHeader);
  L.f = al(L.hist + cap * (8 + 8 + 4));
  L.z = al(L.f + plane * tsize(B->dtype));
  L.total = L.z + (size_t)pd.nbands * plane * zsize(B->z_store);
  return L;
}

}  // namespace

extern "C" {

int mlba_state_size(mlba_ctx* c, size_t* bytes) {
  if (!c || !bytes) return MLBA_E_INVAL;
  *bytes = state_layout(c->b).total;
  return MLBA_OK;
}

int mlba_get_state(mlba_ctx* c, void* blob, size_t bytes) {
  if (!c || !blob) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const StateLayout L = state_layout(B);
  if (bytes < L.total) return MLBA_E_INVAL;
  const Prob& pd = B->hp[0].pd;
  State st;
  CK(cudaMemcpyAsync(&st, &B->d_states[0], sizeof(State), cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  unsigned char* out = static_cast<unsigned char*>(blob);
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = STATE_MAGIC; h.version = STATE_VERSION;
  h.n = pd.n; h.nf = pd.nf; h.p = pd.p; h.bc = pd.bc; h.nbands = pd.nbands;
  h.dtype = B->dtype; h.z_store = B->z_store; h.max_iter = pd.max_iter;
  header_params(pd, h);
  h.iter = st.iter; h.stopped = st.stopped; h.stop_iter = st.stop_iter; h.status = st.status;
  h.nres = st.nres; h.beta_last = st.beta_last;
  h.resnorm = st.resnorm; h.alpha_n = st.alpha_n; h.nb = st.nb; h.qn = st.qn;
  std::memcpy(out, &h, sizeof(h));
  const size_t cap = (size_t)pd.max_iter + 2;
  CK(cudaMemcpy(out + L.hist, pd.hist_res, cap * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out + L.hist + cap * 8, pd.hist_alpha, cap * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out + L.hist + cap * 16, pd.hist_beta, cap * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out + L.f, pd.buf[SL_F], (size_t)pd.nf * pd.nf * tsize(B->dtype),
                cudaMemcpyDeviceToHost));
  return mlba_get_z(c, out + L.z, 0);
}

int mlba_set_state(mlba_ctx* c, const void* blob, size_t bytes) {
  if (!c || !blob) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const StateLayout L = state_layout(B);
  if (bytes < L.total) return MLBA_E_INVAL;
  const Prob& pd = B->hp[0].pd;
  const unsigned char* in = static_cast<const unsigned char*>(blob);
  StateHeader h, mine;
  std::memcpy(&h, in, sizeof(h));
  std::memset(&mine, 0, sizeof(mine));
  header_params(pd, mine);
  if (!same_params(h, mine)) return MLBA_E_INVAL;
  if (h.magic != STATE_MAGIC || h.version != STATE_VERSION || h.n != pd.n || h.nf != pd.nf ||
      h.p != pd.p || h.bc != pd.bc || h.nbands != pd.nbands || h.dtype != B->dtype ||
      h.z_store != B->z_store || h.max_iter != pd.max_iter || h.iter < 0 || h.iter > pd.max_iter ||
      h.nres < 0 || h.nres > pd.max_iter + 2)
    return MLBA_E_INVAL;
  CK(cudaStreamSynchronize(B->stream));
  const size_t cap = (size_t)pd.max_iter + 2;
  CK(cudaMemcpy(pd.hist_res, in + L.hist, cap * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pd.hist_alpha, in + L.hist + cap * 8, cap * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pd.hist_beta, in + L.hist + cap * 16, cap * 4, cudaMemcpyHostToDevice));
  const size_t plane = (size_t)pd.nf * pd.nf;
  CK(cudaMemcpy(pd.buf[SL_F], in + L.f, plane * tsize(B->dtype), cudaMemcpyHostToDevice));
  // z^iter lives in the ping-pong buffer the next frame step reads
  const size_t es = zsize(B->z_store);
  const size_t zbytes = (size_t)pd.nbands * plane * es;
  void* zdst = pd.z[h.iter & 1];
  if (!z_grouped(pd.levels)) {
    CK(cudaMemcpy(zdst, in + L.z, zbytes, cudaMemcpyHostToDevice));
  } else {
    std::vector<unsigned char> g(zbytes);
    for (int b = 0; b < pd.nbands; ++b)
      for (size_t q = 0; q < plane; ++q)
        std::memcpy(g.data() + z_index(b, (int)(q / pd.nf), (int)(q % pd.nf), pd.levels, pd.nf) * es,
                    in + L.z + ((size_t)b * plane + q) * es, es);
    CK(cudaMemcpy(zdst, g.data(), zbytes, cudaMemcpyHostToDevice));
  }
  State st = initial_state(pd);
  st.iter = h.iter; st.stopped = h.stopped; st.stop_iter = h.stop_iter; st.status = h.status;
  st.nres = h.nres; st.beta_last = h.beta_last;
  st.resnorm = h.resnorm; st.alpha_n = h.alpha_n; st.nb = h.nb; st.qn = h.qn;
  CK(cudaMemcpy(&B->d_states[0], &st, sizeof(State), cudaMemcpyHostToDevice));
  return MLBA_OK;
}

void mlba_destroy(mlba_ctx* c) {
  if (!c) return;
  destroy_batch(c->b);
  delete c;
}

// ---- operator entry points ---------------------------------------------------
}  // extern "C"

namespace {
// A f (adj = 0) or A^T t / A' t (adj = 1) of a problem on the FFT blur path,
// input in SL_AUX0: the result lands in SL_AUX1 (n x n) or, for the full
// correlation of a BC / rectangular problem, in SL_V
template <typename T>
void op_fc(mlba_batch* B, int adj) {
  const Prob* P = B->d_probs;
  State* S = B->d_opstates;
  cudaStream_t s = B->stream;
  const ItemList& pad = adj ? B->fc_pad_a : B->fc_pad_f;
  const ItemList& rows = adj ? B->fc_rows_a : B->fc_rows_f;
  const ItemList& cols = adj ? B->fc_cols_a : B->fc_cols_f;
  launch_fc_pad<T>(P, S, pad.dev, pad.count, adj, SL_AUX0, s);
  launch_rows_fwd<T>(P, S, rows.dev, rows.count, SL_R, 0, B->smem_fft, s);
  launch_cols<T>(P, S, cols.dev, cols.count, COL_OP, 0, 1.0, W_TIKH, B->smem_fft, s);
  launch_rows_inv<T>(P, S, rows.dev, rows.count, SL_T, 0, B->smem_fft, s);
  if (!adj) launch_fc_out<T>(P, S, B->fc_out_r.dev, B->fc_out_r.count, FC_STORE_MODE, 0, SL_AUX1, s);
  else if (B->fc_out_u.count) launch_fc_out<T>(P, S, B->fc_out_u.dev, B->fc_out_u.count, FC_STORE_MODE, 1, SL_AUX1, s);
  else launch_fc_out<T>(P, S, B->fc_out_v.dev, B->fc_out_v.count, FC_CORR_MODE, 1, SL_V, s);
}
}  // namespace

extern "C" {

int mlba_op_blur(mlba_ctx* c, const void* f, void* out, int on_device) {
  if (!c) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  const size_t ts = tsize(B->dtype);
  int rc = copy_in(B, pd.buf[SL_AUX0], f, (size_t)pd.nf * pd.nf * ts, on_device);
  if (rc != MLBA_OK) return rc;
  if (reset_opstates(B) != MLBA_OK) return MLBA_E_CUDA;
  if (pd.fc) {
    if (B->dtype == MLBA_F64) op_fc<double>(B, 0); else op_fc<float>(B, 0);
    CK(cudaGetLastError());
    return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
  }
  if (B->dtype == MLBA_F64)
    launch_stencil<double>(ST_FWD_STORE, B->d_probs, B->d_opstates, B->blur.dev, B->blur.count,
                           SL_AUX0, SL_AUX1, SL_AUX1, 0, B->smem_stencil, B->stream);
  else
    launch_stencil<float>(ST_FWD_STORE, B->d_probs, B->d_opstates, B->blur.dev, B->blur.count,
                          SL_AUX0, SL_AUX1, SL_AUX1, 0, B->smem_stencil, B->stream);
  CK(cudaGetLastError());
  return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
}

int mlba_op_blur_adjoint(mlba_ctx* c, const void* t, void* out, int on_device) {
  if (!c) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  const size_t ts = tsize(B->dtype);
  int rc = copy_in(B, pd.buf[SL_AUX0], t, (size_t)pd.n * pd.n * ts, on_device);
  if (rc != MLBA_OK) return rc;
  if (reset_opstates(B) != MLBA_OK) return MLBA_E_CUDA;
  if (pd.fc) {
    if (B->dtype == MLBA_F64) op_fc<double>(B, 1); else op_fc<float>(B, 1);
    CK(cudaGetLastError());
    if (pd.bc == BC_AR) return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
    if (pd.bc != BC_RECT) {
      if (B->dtype == MLBA_F64) launch_vec<double>(VEC_FOLD, B->d_probs, B->d_opstates, B->vec_all.dev, B->vec_all.count, 0, B->stream);
      else launch_vec<float>(VEC_FOLD, B->d_probs, B->d_opstates, B->vec_all.dev, B->vec_all.count, 0, B->stream);
      CK(cudaGetLastError());
      return copy_out(B, out, pd.buf[SL_U], (size_t)pd.n * pd.n * ts, on_device);
    }
    return copy_out(B, out, pd.buf[SL_V], (size_t)pd.nf * pd.nf * ts, on_device);
  }
  if (pd.bc == BC_AR) {
    // the reblurring matrix A' (Section 2.2), n x n
    if (B->dtype == MLBA_F64)
      launch_stencil<double>(ST_REBLUR, B->d_probs, B->d_opstates, B->blur.dev, B->blur.count,
                             SL_AUX0, SL_AUX1, SL_AUX1, 0, B->smem_stencil, B->stream);
    else
      launch_stencil<float>(ST_REBLUR, B->d_probs, B->d_opstates, B->blur.dev, B->blur.count,
                            SL_AUX0, SL_AUX1, SL_AUX1, 0, B->smem_stencil, B->stream);
    CK(cudaGetLastError());
    return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
  }
  if (B->dtype == MLBA_F64) {
    launch_stencil<double>(ST_CORR, B->d_probs, B->d_opstates, B->corr_all.dev, B->corr_all.count,
                           SL_AUX0, SL_V, SL_V, 0, B->smem_stencil, B->stream);
    if (pd.bc != BC_RECT) launch_vec<double>(VEC_FOLD, B->d_probs, B->d_opstates, B->vec_all.dev, B->vec_all.count, 0, B->stream);
  } else {
    launch_stencil<float>(ST_CORR, B->d_probs, B->d_opstates, B->corr_all.dev, B->corr_all.count,
                          SL_AUX0, SL_V, SL_V, 0, B->smem_stencil, B->stream);
    if (pd.bc != BC_RECT) launch_vec<float>(VEC_FOLD, B->d_probs, B->d_opstates, B->vec_all.dev, B->vec_all.count, 0, B->stream);
  }
  CK(cudaGetLastError());
  const void* src = pd.bc == BC_RECT ? pd.buf[SL_V] : pd.buf[SL_U];
  return copy_out(B, out, src, (size_t)pd.nf * pd.nf * ts, on_device);
}

int mlba_op_precond(mlba_ctx* c, const void* r, void* out, double alpha, int which, int on_device) {
  if (!c || !(alpha > 0.0) || which < 0 || which > 1) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  if (pd.transform == TR_NONE) return MLBA_E_INVAL;
  const size_t ts = tsize(B->dtype);
  int rc = copy_in(B, pd.buf[SL_AUX0], r, (size_t)pd.n * pd.n * ts, on_device);
  if (rc != MLBA_OK) return rc;
  if (reset_opstates(B) != MLBA_OK) return MLBA_E_CUDA;
  if (pd.transform == TR_AR) {
    if (B->dtype == MLBA_F64) {
      launch_ar_rows<double>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, 0, B->smem_fft, B->stream);
      launch_ar_cols<double>(B->d_probs, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_OP, 0, alpha, which, B->smem_fft, B->stream);
      launch_ar_rows<double>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX1, 1, 0, B->smem_fft, B->stream);
    } else {
      launch_ar_rows<float>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, 0, B->smem_fft, B->stream);
      launch_ar_cols<float>(B->d_probs, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_OP, 0, alpha, which, B->smem_fft, B->stream);
      launch_ar_rows<float>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX1, 1, 0, B->smem_fft, B->stream);
    }
    CK(cudaGetLastError());
    return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
  }
  if (B->dtype == MLBA_F64) {
    launch_rows_fwd<double>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, B->smem_fft, B->stream);
    launch_cols<double>(B->d_probs, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_OP, 0, alpha, which, B->smem_fft, B->stream);
    launch_rows_inv<double>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX1, 0, B->smem_fft, B->stream);
  } else {
    launch_rows_fwd<float>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, B->smem_fft, B->stream);
    launch_cols<float>(B->d_probs, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_OP, 0, alpha, which, B->smem_fft, B->stream);
    launch_rows_inv<float>(B->d_probs, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX1, 0, B->smem_fft, B->stream);
  }
  CK(cudaGetLastError());
  return copy_out(B, out, pd.buf[SL_AUX1], (size_t)pd.n * pd.n * ts, on_device);
}

int mlba_op_frame(mlba_ctx* c, const void* z_in, const void* u, void* z_out, void* f, double mu,
                  int on_device) {
  if (!c || !z_in || !u || !z_out || !f || !(mu >= 0.0)) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  const size_t ts = tsize(B->dtype);
  const size_t zbytes = (size_t)pd.nbands * pd.nf * pd.nf * zsize(B->z_store);
  const size_t fbytes = (size_t)pd.nf * pd.nf * ts;
  void *dzi = nullptr, *dzo = nullptr;
  if (on_device) { dzi = const_cast<void*>(z_in); dzo = z_out; }
  else {
    CK(cudaMalloc(&dzi, zbytes));
    CK(cudaMalloc(&dzo, zbytes));
    CK(cudaMemcpyAsync(dzi, z_in, zbytes, cudaMemcpyHostToDevice, B->stream));
  }
  // the kernel works on grouped z (L <= 2): convert the caller's band-major
  // planes into scratch copies and back
  const bool grouped = z_grouped(pd.levels);
  const int es = (int)zsize(B->z_store);
  void *gzi = nullptr, *gzo = nullptr;
  if (grouped) {
    CK(cudaMalloc(&gzi, zbytes));
    CK(cudaMalloc(&gzo, zbytes));
    launch_z_layout(gzi, dzi, pd.levels, pd.nf, es, 1, B->stream);
  }
  void* kzi = grouped ? gzi : dzi;
  void* kzo = grouped ? gzo : dzo;
  int rc = copy_in(B, pd.buf[SL_AUX0], u, fbytes, on_device);
  if (rc != MLBA_OK) return rc;
  if (reset_opstates(B) != MLBA_OK) return MLBA_E_CUDA;
  if (B->dtype == MLBA_F64)
    launch_frame<double, double>(B->d_probs, B->d_opstates, B->frame.dev, B->frame.count, B->frame.sec, SL_AUX0, SL_AUX1, kzi, kzo, mu, B->levels, B->frame_shape, B->stream);
  else if (B->z_store == MLBA_BF16)
    launch_frame<float, __nv_bfloat16>(B->d_probs, B->d_opstates, B->frame.dev, B->frame.count, B->frame.sec, SL_AUX0, SL_AUX1, kzi, kzo, mu, B->levels, B->frame_shape, B->stream);
  else
    launch_frame<float, float>(B->d_probs, B->d_opstates, B->frame.dev, B->frame.count, B->frame.sec, SL_AUX0, SL_AUX1, kzi, kzo, mu, B->levels, B->frame_shape, B->stream);
  CK(cudaGetLastError());
  if (grouped) {
    launch_z_layout(dzo, gzo, pd.levels, pd.nf, es, 0, B->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(B->stream));
    cudaFree(gzi);
    cudaFree(gzo);
  }
  rc = copy_out(B, f, pd.buf[SL_AUX1], fbytes, on_device);
  if (rc != MLBA_OK) return rc;
  if (!on_device) {
    CK(cudaMemcpyAsync(z_out, dzo, zbytes, cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    cudaFree(dzi);
    cudaFree(dzo);
  }
  return MLBA_OK;
}

int mlba_op_ns_alpha(mlba_ctx* c, const void* r, double qn, double* alpha_out, int on_device) {
  if (!c || !alpha_out || !(qn > 0.0 && qn < 1.0)) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  if (pd.transform == TR_NONE || pd.transform == TR_AR) return MLBA_E_INVAL;
  const size_t ts = tsize(B->dtype);
  int rc = copy_in(B, pd.buf[SL_AUX0], r, (size_t)pd.n * pd.n * ts, on_device);
  if (rc != MLBA_OK) return rc;
  // op state: Newton armed at log(alpha) = 0
  State s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.ns_active = 1; s0.qn = qn; s0.nb = 0.0; s0.nb_lo = -INFINITY; s0.nb_hi = INFINITY;
  s0.iter = 0; s0.stop_iter = -1;
  CK(cudaMemcpyAsync(B->d_opstates, &s0, sizeof(State), cudaMemcpyHostToDevice, B->stream));
  // a temporary descriptor with the nonstationary flag set and no floor
  Prob tmp = pd;
  tmp.ns = 1;
  tmp.bc = (pd.bc == BC_RECT) ? BC_PERIODIC : pd.bc;   // no rectangular floor here
  tmp.max_iter = -1;                                    // no history writes
  Prob* dtmp = nullptr;
  CK(cudaMalloc(&dtmp, sizeof(Prob)));
  CK(cudaMemcpyAsync(dtmp, &tmp, sizeof(Prob), cudaMemcpyHostToDevice, B->stream));
  if (B->dtype == MLBA_F64) {
    launch_rows_fwd<double>(dtmp, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, B->smem_fft, B->stream);
    launch_cols<double>(dtmp, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_FWD, 0, 0.0, 0, B->smem_fft, B->stream);
    launch_spec<double>(dtmp, B->d_opstates, B->spec_all.dev, B->spec_all.count, 1, B->stream);
    for (int k = 1; k < 60; ++k) launch_spec<double>(dtmp, B->d_opstates, B->spec_all.dev, B->spec_all.count, 0, B->stream);
  } else {
    launch_rows_fwd<float>(dtmp, B->d_opstates, B->rows_all.dev, B->rows_all.count, SL_AUX0, 0, B->smem_fft, B->stream);
    launch_cols<float>(dtmp, B->d_opstates, B->cols_all.dev, B->cols_all.count, COL_FWD, 0, 0.0, 0, B->smem_fft, B->stream);
    launch_spec<float>(dtmp, B->d_opstates, B->spec_all.dev, B->spec_all.count, 1, B->stream);
    for (int k = 1; k < 60; ++k) launch_spec<float>(dtmp, B->d_opstates, B->spec_all.dev, B->spec_all.count, 0, B->stream);
  }
  CK(cudaGetLastError());
  State s1;
  CK(cudaMemcpyAsync(&s1, B->d_opstates, sizeof(State), cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  cudaFree(dtmp);
  *alpha_out = s1.alpha_n;
  return MLBA_OK;
}

int mlba_op_spectrum(mlba_ctx* c, double* out, int* rows, int* cols, int* is_complex) {
  if (!c || !out) return MLBA_E_INVAL;
  mlba_batch* B = c->b;
  const Prob& pd = B->hp[0].pd;
  if (pd.transform == TR_NONE) return MLBA_E_INVAL;
  const bool dct = pd.transform == TR_DCT || pd.transform == TR_AR;   // real spectra
  const size_t W = dct ? pd.n : pd.half;
  const int comps = dct ? 1 : 2;
  const size_t cnt = spec_elems(pd) * comps;
  std::vector<unsigned char> tmp(cnt * tsize(B->dtype));
  CK(cudaMemcpy(tmp.data(), pd.lam, tmp.size(), cudaMemcpyDeviceToHost));
  // undo the column blocking: (k1, k2) lives at (k2 / cb) n cb + k1 cb + k2 % cb
  const size_t cb = pd.cb;
  for (size_t k1 = 0; k1 < (size_t)pd.n; ++k1)
    for (size_t k2 = 0; k2 < W; ++k2)
      for (int q = 0; q < comps; ++q) {
        const size_t src = ((k2 / cb) * pd.n * cb + k1 * cb + k2 % cb) * comps + q;
        out[(k1 * W + k2) * comps + q] = B->dtype == MLBA_F64
            ? reinterpret_cast<double*>(tmp.data())[src]
            : (double)reinterpret_cast<float*>(tmp.data())[src];
      }
  if (rows) *rows = pd.n;
  if (cols) *cols = (int)W;
  if (is_complex) *is_complex = dct ? 0 : 1;
  return MLBA_OK;
}

}  // extern "C"
