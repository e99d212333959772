// mlba_launch.h — host-side launchers of the batched MLBA kernels.
#pragma once
#include <cuda_runtime.h>
#include "mlba_internal.cuh"

namespace mlba {

// stencil modes (k_stencil.cu)
enum {
  ST_FWD_RESID = 0,   // dst = g - A src ; ||dst||^2 -> iteration bookkeeping (stop rule)
  ST_FWD_STORE = 1,   // dst = A src
  ST_FWD_PCGQ = 2,    // dst = A src + alpha aux ; <aux, dst> -> PCG step length
  ST_CORR = 3,        // dst (ne x ne) = full correlation of src (n x n, zero padded)
  ST_REBLUR = 4       // dst (n x n) = A' src: correlation of the antireflectively padded src
                      // (the reblurring matrix of Section 2.2; default dst U)
};
// FFT-convolution blur path (k_stencil.cu): pad a convolution entry's input,
// and move its output to the problem (residual with the stop rule, A f or A' t
// stored n x n, or the (n+p-1)^2 correlation V)
enum { FC_RESID_MODE = 0, FC_STORE_MODE = 1, FC_CORR_MODE = 2 };
template <typename T>
void launch_fc_pad(const Prob* probs, State* states, const int2* items, int nitems, int adj,
                   int src_slot, cudaStream_t s);
template <typename T>
void launch_fc_out(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                   int adj, int dst_slot, cudaStream_t s);
// balanced formulation: u <- f + u before the framelet step (k_stencil.cu)
template <typename T>
void launch_balance(const Prob* probs, State* states, const int2* items, int nitems, cudaStream_t s);
// vector kernels (k_stencil.cu)
enum {
  VEC_FOLD = 0,       // U = BC fold of V
  VEC_PCG_INIT = 1,   // PX = 0, PRES = R
  VEC_PCG_RHO0 = 2,   // rho0 = <PRES, PZ>, PP = PZ
  VEC_PCG_AXPY = 3,   // PX += a PP, PRES -= a PQ
  VEC_PCG_RHO = 4,    // rho = <PRES, PZ>, convergence test
  VEC_PCG_PUPD = 5,   // PP = PZ + beta PP
  VEC_PCG_FINISH = 6  // T = PX
};
// column-pass modes (k_fft.cu)
enum {
  COL_FUSED = 0,      // forward, weight (stationary alpha), inverse
  COL_FWD = 1,        // forward only, spectrum kept in S (4-NS)
  COL_NS_INV = 2,     // weight with alpha_n, inverse (4-NS)
  COL_OP = 3          // forward, weight with the operator's alpha / kind, inverse
};
enum { W_INV = 0, W_TIKH = 1 };

constexpr int STENCIL_THREADS = 128;
constexpr int VEC_THREADS = 256;
constexpr int VEC_PER_THREAD = 8;
constexpr int TR_CAP = 4096;          // complex values held by one transform CTA
constexpr int FRAME_SHAPES = 8;      // tile shapes of the L <= 2 framelet kernel (k_frame.cu)
constexpr int LV_NWR = 1;            // warps per CTA of the per-level framelet kernel (L >= 3; 1, 2, 4 measured)
constexpr int LP_THREADS = 256, LP_PER = 4;   // low-pass chain kernel (L >= 3)
constexpr int FRAME_SECTIONS = 2 + 4;         // fold, low-pass, up to four levels
constexpr int SPEC_THREADS = 256;    // alpha_n solve (k_fft.cu)
constexpr int SPEC_PER_THREAD = 32;
constexpr int SPEC_SUMS = 17;        // block sums of the bracketing pass (2 x 8 candidates + 1)

template <typename T>
void launch_stencil(int mode, const Prob* probs, State* states, const int2* items, int nitems,
                    int src, int dst, int aux, int pcg, size_t smem, cudaStream_t s);
template <typename T>
void launch_vec(int mode, const Prob* probs, State* states, const int2* items, int nitems,
                int pcg, cudaStream_t s);
template <typename T>
void launch_rows_fwd(const Prob* probs, State* states, const int2* items, int nitems, int src,
                     int pcg, size_t smem, cudaStream_t s);
template <typename T>
void launch_cols(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                 int pcg, double op_alpha, int op_kind, size_t smem, cudaStream_t s);
template <typename T>
void launch_rows_inv(const Prob* probs, State* states, const int2* items, int nitems, int dst,
                     int pcg, size_t smem, cudaStream_t s);
template <typename T>
void launch_spec(const Prob* probs, State* states, const int2* items, int nitems, int cand,
                 cudaStream_t s);
// antireflective transform passes (k_fft.cu): rows (inv = 0: T^{-1} of
// buf[slot] into S; inv = 1: T of S into buf[slot]) and the column pass
// (T^{-1}, weight, T; mode COL_FUSED or COL_OP)
template <typename T>
void launch_ar_rows(const Prob* probs, State* states, const int2* items, int nitems, int slot,
                    int inv, int pcg, size_t smem, cudaStream_t s);
template <typename T>
void launch_ar_cols(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                    int pcg, double op_alpha, int op_kind, size_t smem, cudaStream_t s);
void launch_spectrum_setup(int transform, int n, int p, int half, int cb, const double* q_dev,
                           const double* tab_dev, void* lam, void* sigT, int is_double,
                           cudaStream_t s);
// The framelet step.  levels <= 2: one launch of the fused sweep over
// `items` in tile shape `shape`.  levels >= 3: the item list holds sections
// whose (offset, count) pairs `sec` gives: the BC fold of the correlation
// (VEC_FOLD items, skipped when u_slot >= 0), the low-pass chain (one block
// per output row), then the level kernels of level L, L-1, ..., 1.
template <typename T, typename TZ>
void launch_frame(const Prob* probs, State* states, const int2* items, int nitems, const int* sec,
                  int u_slot, int f_slot, const void* zin, void* zout, double op_mu, int levels,
                  int shape, cudaStream_t s);
int frame_tiles(int nf, int levels, int shape);   // CTAs of the fused sweep for one problem (L <= 2)
int lev_tiles(int nf, int lev);                   // CTAs of one level kernel (L >= 3)
int lowpass_blocks(int nf);                       // CTAs of one low-pass launch (L >= 3)
void frame_shape(int shape, int* tile_x, int* tile_y, int* prefetch);
bool is_frame_kernel(const void* func);  // func is one of the framelet-update kernels
int stencil_tiles(int outN);             // CTAs of the stencil for an outN x outN output
// z layout: the 8 high-pass bands of a level contiguous per position, in
// the polyphase order of the level's dilation for L >= 3 (z_index);
// conversion to / from band-major planes
bool z_grouped(int levels);
void launch_z_layout(void* dst, const void* src, int levels, int nf, int elem_bytes,
                     int to_grouped, cudaStream_t s);
template <typename T, typename TZ>
cudaError_t frame_set_smem();

// Persistent step kernel (k_persist.cu): a stage of the step and its items
enum { PS_RESID = 0, PS_CORR, PS_REBLUR, PS_ROWS_FWD, PS_COLS_FUSED, PS_COLS_FWD, PS_SPEC,
       PS_COLS_NSINV, PS_ROWS_INV, PS_BALANCE, PS_FRAME };
struct PersistStage {
  int kind, count;
  const int2* items;
  int sync;            // 1: a grid barrier follows (the next stage reads what this one wrote)
  int pad;
};
size_t persist_smem(int dtype_bytes, int zs_bytes, int levels, size_t smem_stencil, size_t smem_fft,
                    int* stencil_slot, int* frame_slot);
const void* persist_func(int zs_bytes, int levels);
cudaError_t persist_graph(int zs_bytes, int levels, int grid, size_t smem, const Prob* probs,
                          State* states, int nprob, const PersistStage* stages, int nst, int ksteps,
                          void* ctl, unsigned long long spin_ns, int stencil_slot, int frame_slot,
                          cudaGraph_t* g, cudaGraphNode_t* knode);
cudaError_t persist_graph_set_k(cudaGraphExec_t x, cudaGraphNode_t knode, int zs_bytes, int levels,
                                int grid, size_t smem, const Prob* probs, State* states, int nprob,
                                const PersistStage* stages, int nst, int ksteps, void* ctl,
                                unsigned long long spin_ns, int stencil_slot, int frame_slot);
size_t persist_ctl_bytes();
int persist_threads();
template <typename T>
cudaError_t stencil_set_smem(size_t bytes);
template <typename T>
cudaError_t fft_set_smem(size_t bytes);

}  // namespace mlba
