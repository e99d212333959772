// mlba_internal.cuh — device-side data model shared by the kernels and the
// host runtime of the MLBA library.  Every kernel is batched: a launch walks
// an item list of (problem, block) pairs so that one launch serves all
// problems of a batch (a single problem is a batch of one).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mlba {

// ----------------------------------------------------------------------------
// enumerations mirrored from include/mlba.h
enum { BC_ZERO = 0, BC_PERIODIC = 1, BC_REFLECTIVE = 2, BC_RECT = 3, BC_AR = 4 };
enum { P_NONE = 0, P_BCCB = 1, P_KRYLOV = 2, P_SYM = 3, P_TIKH = 4, P_TIKH_NS = 5 };
enum { TR_NONE = 0, TR_DFT = 1, TR_DCT = 2, TR_AR = 3 };

// per-problem buffer slots; kernels pick their operands by slot so that the
// same kernel serves the main loop, the PCG of Algorithm 2 and the operator
// entry points
enum Slot {
  SL_G = 0,   // observed image g (n x n)
  SL_F,       // current image f (Nf x Nf)
  SL_R,       // residual r (n x n)
  SL_T,       // preconditioned residual t (n x n)
  SL_V,       // full correlation of t on the extended (n+p-1)^2 domain
  SL_U,       // BC-folded A^T t (n x n); PCG work
  SL_S,       // transform work array (column-blocked spectrum, see Prob::cb)
  SL_PX, SL_PRES, SL_PP, SL_PQ, SL_PZ,  // PCG vectors (n x n)
  SL_AUX0, SL_AUX1,                     // operator entry-point scratch (Nf x Nf)
  NSLOT
};

constexpr int MAX_STAGES = 24;
constexpr int MAX_LEVELS = 4;

// Constant description of one problem (device copy lives in a table).
struct Prob {
  int n, p, c, nf, ne, half;     // half = n/2+1
  int sidx;          // index of the State this entry answers to: its own, or for a
                     // convolution entry (FFT blur path) the problem it serves
  int fc;            // problem: 1 = A and A^T by FFT convolution (the entries below)
  int fc_sh[2];      // problem: table indices of its forward / adjoint convolution entries
  int balanced;      // 1: the balanced formulation, x = S_mu(W (f + u)): u is replaced by
                     // f + u before the framelet step and z_in by zeros (z0)
  int bc, precond, transform, levels, nbands;
  int ns;            // nonstationary alpha (4-NS)
  int use_adj;       // 1: u = A^T t ; 0: u = t (Algorithm 4 forms)
  int sep;           // rank-one PSF: separable stencils
  int ntaps;         // nonzero taps of the PSF
  int nruns, nrw;    // PSF column runs and their packed weights (general PSF)
  int max_iter, stop, pcg_max;
  int nfft;          // FFT length: n (DFT, DCT) or 2(n - 1) (antireflective transform)
  int nstage;        // FFT plan of length nfft
  int radix[MAX_STAGES];
  int nr16, r2, nr3, nr5;   // the same plan: radix-16 passes, one 8/4/2 pass, 3s, 5s,
  int nrany;                // then the prime factors above 5 (direct-sum passes)
  // per-list block counts (reductions need them)
  int nblk_blur, nblk_corr, nblk_rows, nblk_cols, nblk_spec, nblk_vec;
  int row_g, col_g;  // transforms per CTA in the row / column passes
  int cb;            // spectrum column block: col_g complex columns (DFT) or
                     // 2 col_g real columns (DCT); block j holds columns
                     // [j cb, (j+1) cb) as n rows of cb contiguous elements;
                     // there are nblk_cols blocks, the last one may be padded
  double mu, alpha, gamma, delta, q, rho, tau, pcg_tol;
  void* buf[NSLOT];
  void* z[2];        // ping-pong Bregman variable
  void* z0;          // balanced formulation: zeros read in place of z_in
  void* w;           // |lambda|^2 in T precision, column-blocked like S
  void* pw;          // 4-NS: weighted power |orthonormal coefficient of r|^2 per
                     // spectral value, T, blocked like S (0 on padding); written by
                     // the bracketing pass, read by the Halley passes
  void* lam;         // spectrum of C (real for DCT, complex half for DFT), T, blocked
  void* lp;          // L >= 3: low-pass chain c_1 .. c_{L-1} (nf x nf planes, T)
  void* sy;          // L >= 3: synthesis partials s_1 .. s_{L-1} (nf x nf planes, T)
  void* tw;          // exp(-2 pi i k/nfft), k < nfft   (T2)
  void* dtw;         // exp(-i pi k/(2n)), k < n  (T2)
  int4* tap_runs;     // per nonzero PSF column b: (b, lo, hi, offset of H[lo..hi][b] in tap_w)
  void* tap_w;        // packed run weights, T precision: nrw in PSF order, then nrw with
                      // every run reversed
  void* hy; void* hx;                      // separable factors (length p)
  double* partial;   // reduction partials (capacity per problem)
  double* hist_res; double* hist_alpha; int* hist_beta;  // history, max_iter+2
};

// Mutable per-problem state (device).
struct State {
  int iter;          // z-updates done (f = f^iter)
  int stopped;       // no more updates
  int stop_iter;     // first n with the rule satisfied, -1 if none
  int status;        // 0 or MLBA_E_DIVERGED
  int nres;          // residuals computed
  unsigned int counter;  // last-block reduction counter
  int ns_active;     // 4-NS: alpha_n being solved this iteration
  int nconv;         // 4-NS Newton converged
  int npass;
  int nphase;        // 4-NS: 0 = bracketing pass pending, 1 = Newton
  int pdone, psteps; // PCG
  int beta_last;
  double resnorm, alpha_n, qn;
  double nb, nb_lo, nb_hi;     // Newton on log(alpha)
  double ea;                   // exp(nb), set with nb (before the rectangular floor)
  double prho, prho0, pa, pbeta;
};

// ----------------------------------------------------------------------------
// small helpers

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T2, typename T>
__host__ __device__ __forceinline__ T2 mk2(T a, T b) { T2 r; r.x = a; r.y = b; return r; }

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { a.x += b.x; a.y += b.y; return a; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { a.y = -a.y; return a; }

// storage conversions for z
__device__ __forceinline__ float ld_z(const float* p) { return *p; }
__device__ __forceinline__ double ld_z(const double* p) { return *p; }
__device__ __forceinline__ float ld_z(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st_z(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_z(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_z(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Table 1 boundary map: FOV index copied by extended index e, or -1 (zero).
__device__ __forceinline__ int bc_map(int e, int n, int bc) {
  if (e >= 0 && e < n) return e;
  if (bc == BC_ZERO) return -1;
  if (bc == BC_PERIODIC) { int q = e % n; return q < 0 ? q + n : q; }
  int m2 = 2 * n;
  int q = e % m2; if (q < 0) q += m2;
  return q < n ? q : m2 - 1 - q;
}

// half-sample symmetric reflection used by the framelets; *odd tells whether
// an odd number of mirrorings happened (antisymmetric bands flip sign)
__device__ __forceinline__ int refl_half(int e, int n, int* odd) {
  int m2 = 2 * n;
  int q = e % m2; if (q < 0) q += m2;
  // e = q + k*2n; each period contains two mirrorings, so parity is that of q >= n
  if (q < n) { *odd = 0; return q; }
  *odd = 1; return m2 - 1 - q;
}

// bring the 128-byte line of p into L2 (no registers, no wait)
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of every 128-byte line of [p, p + bytes) by the threads
// tid = 0 .. nt - 1 of a group
__device__ __forceinline__ void prefetch_range(const void* p, size_t bytes, int tid, int nt) {
  const size_t a0 = reinterpret_cast<size_t>(p) & ~size_t(127);
  const size_t a1 = reinterpret_cast<size_t>(p) + bytes;
  for (size_t a = a0 + (size_t)tid * 128; a < a1; a += (size_t)nt * 128)
    prefetch_l2(reinterpret_cast<const void*>(a));
}

// n / d by a multiply-high: m = floor((2^32 - 1) / d) + 1 gives the exact
// quotient whenever 0 <= n and n d < 2^32 (every index here is below 2^17
// and every divisor at most 8192); d = 1 passes n through
struct FastDiv {
  unsigned m;
  int d;
  __device__ __forceinline__ explicit FastDiv(int dd)
      : m(dd > 1 ? 0xFFFFFFFFu / (unsigned)dd + 1u : 0u), d(dd) {}
  __device__ __forceinline__ int div(int n) const {
    return d == 1 ? n : (int)__umulhi((unsigned)n, m);
  }
};

// Polyphase order of one image axis for a dilation D (a power of two): the
// position x = a + D m (a = x mod D) is stored at S_a + m with S_a =
// a Q + min(a, R), nf = D Q + R, so the D sub-lattices of the axis follow one
// another, each in increasing order (sub-lattice a holds M_a = Q + [a < R]
// positions).  A plane in this order has its rows and its columns permuted
// so; D = 1 is the identity.  A filter with taps D apart then reaches
// neighbouring positions of one sub-lattice.
struct Poly {
  int D, sh, Q, R;
  __host__ __device__ Poly(int nf, int d) : D(d), sh(0), Q(0), R(0) {
    while ((1 << sh) < d) ++sh;
    Q = nf >> sh;
    R = nf - (Q << sh);
  }
  __host__ __device__ int count(int a) const { return Q + (a < R ? 1 : 0); }
  __host__ __device__ int count_max() const { return Q + (R > 0 ? 1 : 0); }
  __host__ __device__ int start(int a) const { return a * Q + (a < R ? a : R); }
  __host__ __device__ int pos(int x) const { return start(x & (D - 1)) + (x >> sh); }
  // x from its position p
  __host__ __device__ int inv(int p) const {
    const int big = R * (Q + 1);
    int a, m;
    if (p < big) { a = p / (Q + 1); m = p - a * (Q + 1); }
    else { const int r = p - big; a = R + r / Q; m = r - (a - R) * Q; }
    return a + (m << sh);
  }
};

// Poly::inv with the two quotients by multiply-high (device code)
struct PolyInv {
  Poly P;
  FastDiv q1, q0;
  int big;
  __device__ __forceinline__ PolyInv(int nf, int d)
      : P(nf, d), q1(P.Q + 1), q0(P.Q > 0 ? P.Q : 1), big(P.R * (P.Q + 1)) {}
  __device__ __forceinline__ int inv(int p) const {
    int a, m;
    if (p < big) { a = q1.div(p); m = p - a * (P.Q + 1); }
    else { const int r = p - big; const int k = q0.div(r); a = P.R + k; m = r - k * P.Q; }
    return a + (m << P.sh);
  }
};

// Internal position of z band b at pixel (y, x): the 8 high-pass bands of
// level l of a position are contiguous at (l - 1) 8 nf^2 + 8 q + (b mod 8),
// the final low-pass band has the plane 8 L nf^2 + q.  q = y nf + x for
// L <= 2; for L >= 3 the planes of level l are in the polyphase order of its
// dilation 2^(l-1) (the low-pass band in that of level L), the order in which
// the per-level kernels sweep them.
__host__ __device__ inline size_t z_index(int b, int y, int x, int levels, int nf) {
  const size_t plane = (size_t)nf * nf;
  const int nb = 8 * levels + 1;
  const int lev = b < nb - 1 ? b / 8 + 1 : levels;
  const Poly P(nf, levels >= 3 ? 1 << (lev - 1) : 1);
  const size_t q = (size_t)P.pos(y) * nf + P.pos(x);
  return b < nb - 1 ? (size_t)(b / 8) * 8 * plane + 8 * q + (b % 8) : (size_t)b * plane + q;
}

// Thread groups a body of work runs on: the whole CTA, or a sub-block of NTS
// threads (whole warps) of a larger CTA with its own hardware barrier `id`
// (1..15; barrier 0 is __syncthreads).  The bodies of the persistent step
// kernel run several stencil or framelet items side by side this way.
struct BlkFull {
  __device__ __forceinline__ int tid() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
template <int NTS>
struct BlkSub {
  int id;
  __device__ __forceinline__ int tid() const { return threadIdx.x % NTS; }
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NTS) : "memory");
  }
};

// block-wide sum of a double (deterministic order) over the NT threads of
// group b; all of them must call
template <int NT, typename BLK>
__device__ __forceinline__ double block_sum_b(double v, double* sh, BLK b) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int t = b.tid();
  int w = t >> 5, l = t & 31;
  b.sync();
  if (l == 0) sh[w] = v;
  b.sync();
  double r = 0.0;
  if (t < 32) {
    r = (t < NT / 32) ? sh[t] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0 of the group
}
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  return block_sum_b<NT>(v, sh, BlkFull{});
}

// block-wide sums of K doubles with one barrier: warp shuffles, then one
// thread per value sums the warp partials in warp order (results in thread 0's
// out[] after the call; every thread must call)
template <int NT, int K>
__device__ __forceinline__ void block_sum_k(double (&v)[K], double (&out)[K], double* sh) {
  constexpr int NW = NT / 32;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * NW + w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = 0; i < NW; ++i) s += sh[k * NW + i];
      out[k] = s;
    }
  }
}

// Last-block reduction: every block of problem `pi` calls this with its K
// partial values (valid in thread 0); the block that arrives last returns
// true with the K totals (summed in block order) in tot[] (valid in thread 0).
// `flag`: one shared int of the group.
template <int NT, int K, typename BLK>
__device__ bool last_block_reduce_b(const Prob& pd, State& st, int blk, int nblk,
                                    const double* vals, double* tot, double* sh, int* flag, BLK b) {
  const int t = b.tid();
  if (t == 0) {
    for (int k = 0; k < K; ++k) pd.partial[(size_t)k * nblk + blk] = vals[k];
    __threadfence();
    unsigned int prev = atomicAdd(&st.counter, 1u);
    *flag = (prev == (unsigned)(nblk - 1));
  }
  b.sync();
  if (!*flag) return false;
  __threadfence();
  for (int k = 0; k < K; ++k) {
    // thread t adds blocks t, t + NT, ... in that order, 4 loads in flight
    const double* pk = pd.partial + (size_t)k * nblk;
    double s = 0.0;
    int i = t;
    for (; i + 3 * NT < nblk; i += 4 * NT) {
      const double a0 = __ldcg(pk + i), a1 = __ldcg(pk + i + NT);
      const double a2 = __ldcg(pk + i + 2 * NT), a3 = __ldcg(pk + i + 3 * NT);
      s += a0; s += a1; s += a2; s += a3;
    }
    for (; i < nblk; i += NT) s += __ldcg(pk + i);
    s = block_sum_b<NT>(s, sh, b);
    if (t == 0) tot[k] = s;
  }
  if (t == 0) st.counter = 0u;
  return true;
}
template <int NT, int K>
__device__ bool last_block_reduce(const Prob& pd, State& st, int blk, int nblk,
                                  const double* vals, double* tot, double* sh) {
  __shared__ int is_last;
  return last_block_reduce_b<NT, K>(pd, st, blk, nblk, vals, tot, sh, &is_last, BlkFull{});
}

// BC fold of the extended correlation: u(a,b) = sum over the padded positions
// that copy (a,b) (transpose of the Table 1 padding).
template <typename T>
__device__ __forceinline__ T fold_fetch(const Prob& pd, const T* V, int a, int b) {
  const int n = pd.n, c = pd.c, ne = pd.ne;
  int cy[3], cx[3], ny = 1, nx = 1;
  cy[0] = a; cx[0] = b;
  if (pd.bc == BC_PERIODIC) {
    if (a + n <= n - 1 + c) cy[ny++] = a + n;
    if (a - n >= -c) cy[ny++] = a - n;
    if (b + n <= n - 1 + c) cx[nx++] = b + n;
    if (b - n >= -c) cx[nx++] = b - n;
  } else if (pd.bc == BC_REFLECTIVE) {
    if (-1 - a >= -c) cy[ny++] = -1 - a;
    if (2 * n - 1 - a <= n - 1 + c) cy[ny++] = 2 * n - 1 - a;
    if (-1 - b >= -c) cx[nx++] = -1 - b;
    if (2 * n - 1 - b <= n - 1 + c) cx[nx++] = 2 * n - 1 - b;
  }
  T s = T(0);
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) s += V[(size_t)(cy[i] + c) * ne + (cx[j] + c)];
  return s;
}

}  // namespace mlba
