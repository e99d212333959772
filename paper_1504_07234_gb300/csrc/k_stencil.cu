// k_stencil.cu — PSF stencils of the blurring operator (Section 2), their
// residual / PCG epilogues, and the elementwise kernels of the Krylov
// preconditioner (Section 4.2).
//
// Blur A (Eq. modeld, Table 1, Eq. Arect): (A f)(i,j) = sum_{dy,dx}
// h(dy,dx) f_ext(i-dy, j-dx), f_ext being f padded by the boundary condition
// (index math only) or, for the rectangular operator, the m x m unknown whose
// field of view is offset by c = (p-1)/2.
// Adjoint: the full correlation V(a,b) = sum h(dy,dx) t0(a-c+dy, b-c+dx) on
// the (n+p-1)^2 extended domain (t zero outside), which is A^T t for the
// rectangular operator; for a boundary condition the fold of V by the
// transpose of the padding gives A^T t (done where u is consumed).
// Antireflective BCs (Section 2.2) pad by 2 F(edge) - F(mirror) instead of a
// copy, and A^T is replaced by the reblurring matrix A': the correlation of
// the antireflectively padded t on the n x n domain.
#include "mlba_internal.cuh"
#include "mlba_launch.h"

namespace mlba {

// stop rule and iteration bookkeeping after ||r^n||^2 is known
// (Eq. discrpr; Algorithm 4-NS and Eq. Alg4_rev_12)
static __device__ void finalize_residual(const Prob& pd, State& st, double sumsq) {
  const int it = st.iter;
  const double rn = sqrt(sumsq);
  st.resnorm = rn;
  if (st.nres < pd.max_iter + 2) pd.hist_res[st.nres] = rn;
  st.nres++;
  if (!isfinite(rn)) { st.status = -5; st.stopped = 1; return; }
  const bool crossed = pd.ns ? (rn <= pd.tau * pd.delta) : (it > 0 && rn <= pd.gamma * pd.delta);
  if (crossed && st.stop_iter < 0) st.stop_iter = it;
  if ((crossed && pd.stop) || it >= pd.max_iter) { st.stopped = 1; return; }
  if (pd.ns) {
    if (!crossed) {
      // q_n = max{q, 2 rho + (1 + rho)/tau_n}, tau_n = ||r^n|| / delta
      const double qn = fmax(pd.q, 2.0 * pd.rho + (1.0 + pd.rho) * pd.delta / rn);
      st.qn = qn;
      st.ns_active = 1;
      st.nconv = 0;
      st.npass = 0;
      st.nphase = 0;
      st.nb_lo = -INFINITY;
      st.nb_hi = INFINITY;
    } else {
      st.ns_active = 0;   // past the discrepancy point alpha_n is kept
      if (it < pd.max_iter + 2) pd.hist_alpha[it] = st.alpha_n;
    }
  }
  st.iter = it + 1;
}

__device__ __forceinline__ bool skip(const State& st, int pcg) {
  return st.stopped || (pcg && st.pdone);
}

// The last R (1..7) taps t .. t + R - 1 of a run from the aligned window
// (slot j holds v[t + j]): v[t + 8 .. t + R + 6] go to R - 1 more registers and
// every index is static, so no value moves and no work is predicated off.
template <int R, typename V, typename W, typename LD, typename FMA>
__device__ __forceinline__ void window_tail(V (&acc)[8], const V (&win)[8], const W* __restrict__ w,
                                            int t, LD ld, FMA fma2) {
  V ext[R > 1 ? R - 1 : 1];
#pragma unroll
  for (int i = 0; i < R - 1; ++i) ext[i] = ld(t + 8 + i);
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const W wt = w[t + u];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int sidx = j + u;
      acc[j] = fma2(sidx < 8 ? win[sidx] : ext[sidx - 8 < R - 1 ? sidx - 8 : 0], wt, acc[j]);
    }
  }
}
template <typename V, typename W, typename LD, typename FMA>
__device__ __forceinline__ void window_tails(V (&acc)[8], const V (&win)[8], const W* __restrict__ w,
                                             int t, int r, LD ld, FMA fma2) {
  switch (r) {
    case 1: window_tail<1>(acc, win, w, t, ld, fma2); break;
    case 2: window_tail<2>(acc, win, w, t, ld, fma2); break;
    case 3: window_tail<3>(acc, win, w, t, ld, fma2); break;
    case 4: window_tail<4>(acc, win, w, t, ld, fma2); break;
    case 5: window_tail<5>(acc, win, w, t, ld, fma2); break;
    case 6: window_tail<6>(acc, win, w, t, ld, fma2); break;
    case 7: window_tail<7>(acc, win, w, t, ld, fma2); break;
    default: break;
  }
}

// acc[j] += sum_t w[t] v[t + j] over a run of len taps, v[i] = base[i * stride]:
// an 8-value window of v.  Whole groups of 8 taps keep the window as a ring
// (slot (i & 7) holds v[i]) so every register index is static and no value
// moves; after them the ring is aligned again (slot j holds v[t + j]) and the
// last len % 8 taps go through window_tail.
template <typename T>
__device__ __forceinline__ void window_run(T (&acc)[8], const T* __restrict__ base, int stride,
                                           const T* __restrict__ w, int len) {
  T win[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) win[j] = base[j * stride];
  int t = 0;
  for (; t + 8 <= len; t += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T wt = w[t + u];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += wt * win[(j + u) & 7];
      // slot u held v[t + u], needed by no later tap: refill with v[t + u + 8]
      if (t + u + 1 < len) win[u] = base[(t + u + 8) * stride];
    }
  }
  window_tails(acc, win, w, t, len - t, [&](int i) { return base[i * stride]; },
               [](T v, T wt, T a) { return a + wt * v; });
}

// asynchronous global -> shared copy of a B-byte chunk (B = 8 or 16, both
// addresses B-aligned) of which the first nbytes come from global memory and
// the rest are zero-filled
template <int B>
__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, int nbytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}

// asynchronous global -> shared copy of one 4- or 8-byte element; !valid
// writes zeros (0 source bytes)
template <int B>
__device__ __forceinline__ void cp_async_zfill(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int src_bytes = valid ? B : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(B),
               "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Table 1 map for an extended index within one period of the image (the
// common case), else the general map
__device__ __forceinline__ int bc_map_near(int e, int n, int bc) {
  if (e >= 0 && e < n) return e;
  if (e >= -n && e < 2 * n) {
    if (bc == BC_ZERO) return -1;
    if (bc == BC_PERIODIC) return e < 0 ? e + n : e - n;
    return e < 0 ? -1 - e : 2 * n - 1 - e;
  }
  return bc_map(e, n, bc);
}

// Pairs of FP32 values: the paired FP32 instructions of sm_100+ do two
// multiply-adds in one; FP64 falls back to two scalar ones.
template <typename T> struct Pair;
template <> struct Pair<float> {
  using type = float2;
  static __device__ __forceinline__ float2 fma(float2 a, float w, float2 acc) {
    return __ffma2_rn(a, make_float2(w, w), acc);
  }
};
template <> struct Pair<double> {
  using type = double2;
  static __device__ __forceinline__ double2 fma(double2 a, double w, double2 acc) {
    return make_double2(::fma(a.x, w, acc.x), ::fma(a.y, w, acc.y));
  }
};

// acc[j] += sum_t w[t] v[t + j] over a run of len taps for pairs of
// neighbouring columns, v[i] = (base[i stride], base[i stride + 1]) (one
// 8-byte or 16-byte load when `aligned`, else two): the same ring / shifting
// window as window_run, on pairs.
template <typename T>
__device__ __forceinline__ void window_run2(typename Pair<T>::type (&acc)[8], const T* __restrict__ base,
                                            int stride, const T* __restrict__ w, int len,
                                            bool aligned) {
  using T2 = typename Pair<T>::type;
  auto ld = [&](int i) -> T2 {
    const T* q = base + i * stride;
    if (aligned) return *reinterpret_cast<const T2*>(q);
    T2 v; v.x = q[0]; v.y = q[1]; return v;
  };
  T2 win[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) win[j] = ld(j);
  int t = 0;
  for (; t + 8 <= len; t += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T wt = w[t + u];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = Pair<T>::fma(win[(j + u) & 7], wt, acc[j]);
      if (t + u + 1 < len) win[u] = ld(t + u + 8);
    }
  }
  window_tails(acc, win, w, t, len - t, ld, [](T2 v, T wt, T2 a) { return Pair<T>::fma(v, wt, a); });
}

// Stencil tile geometry: 64 x 32 outputs per CTA of 128 threads; a thread
// owns two neighbouring columns over 8 rows (16 outputs in registers).  The
// input tile (32 + p - 1) x (64 + p - 1) lives in shared memory with an even
// row pitch (pairs of columns are one 8-byte word when the column is even).
constexpr int ST_TX = 64, ST_TY = 32;
// row pitch of the input tile: a multiple of 16 bytes with room for the
// shift (< 16 bytes) that aligns a row's source to 16 bytes
__host__ __device__ constexpr int st_pitch(int RX, int elem) {
  return (RX + 16 / elem - 1 + 16 / elem - 1) / (16 / elem) * (16 / elem);
}
constexpr int ST_TP = ST_TX + 2;      // row-pass tile pitch (rank-one PSF, p > 33)
constexpr int ST_ROW_ITEMS = 4;       // row-pass items a thread holds in registers (8 RY <= 4 x 128)

#ifndef MLBA_BODIES_ONLY
int stencil_tiles(int outN) { return ((outN + ST_TX - 1) / ST_TX) * ((outN + ST_TY - 1) / ST_TY); }
#endif

// Blur A (Eq. 2 with the Table 1 boundary conditions, or the valid part for
// rectangular A) and the full correlation that A^T is built from, as
// register-window stencils:
//  - general PSF: the taps are grouped by PSF column b into dense runs
//    [lo_b, hi_b] of rows; a thread slides an 8-row window of two input
//    columns down the run, so each tap costs one (or two) shared loads, one
//    broadcast weight and 8 paired FMAs for 16 outputs;
//  - rank-one PSF (h = hy hx^T): a horizontal pass with an 8-value window along
//    the rows into shared memory, then a vertical pass with paired windows.
// Forward (A f)(y, x) = sum_{a,b} H[a][b] f_ext(y + c - a, x + c - b); the
// correlation (ne x ne) is sum_{a,b} H[a][b] t(y - 2c + a, x - 2c + b).
// (FP32: 8 CTAs per SM, 64 registers; the tile of the largest PSF of a batch
// decides how many fit in shared memory)
// One stencil item (tile) on the thread group `blk` of STENCIL_THREADS threads,
// with its shared memory at smraw, 32 doubles of reduction space and one int.
template <typename T, int MODE, typename BLK>
__device__ __forceinline__ void stencil_body(const int2 item, const Prob* __restrict__ probs,
                                             State* __restrict__ states, int src_slot, int dst_slot,
                                             int aux_slot, int pcg, unsigned char* smraw,
                                             double* red, int* flag, BLK blk) {
  using T2 = typename Pair<T>::type;
  const int tid = blk.tid();
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (skip(st, pcg)) return;

  // CORR: correlation weights and run offsets (the full correlation and the
  // reblurring A' of antireflective BCs); ZPAD: the full correlation of the
  // zero-padded t on the (n+p-1)^2 domain
  constexpr bool CORR = (MODE == ST_CORR || MODE == ST_REBLUR);
  constexpr bool ZPAD = (MODE == ST_CORR);
  constexpr int NT = STENCIL_THREADS;
  const int n = pd.n, p = pd.p, c = pd.c;
  const int outN = ZPAD ? pd.ne : n;
  const int tilesX = (outN + ST_TX - 1) / ST_TX;
  const int ty0 = (item.y / tilesX) * ST_TY, tx0 = (item.y % tilesX) * ST_TX;
  const int RY = ST_TY + p - 1, RX = ST_TX + p - 1;
  const int RP = st_pitch(RX, (int)sizeof(T));
  const bool sep = pd.sep != 0;

  // shared memory: weights, column runs (general PSF), input tile, row-pass
  // tile (rank-one PSF)
  const int nw = sep ? 2 * p : pd.nrw;
  T* s_w = reinterpret_cast<T*>(smraw);
  int4* s_runs = reinterpret_cast<int4*>(s_w + ((nw + 3) & ~3));
  T* s_in = reinterpret_cast<T*>(s_runs + (sep ? 0 : pd.nruns));
  T* s_tmp = s_in + RY * RP;

  // src_slot < 0: the per-problem default operand (t, or r for P = I, in the
  // correlation; A^T p for the PCG product: V for rectangular A, U otherwise)
  if (src_slot < 0)
    src_slot = CORR ? (pd.precond == P_NONE ? SL_R : SL_T) : (pd.bc == BC_RECT ? SL_V : SL_U);
  if (MODE == ST_REBLUR && dst_slot < 0) dst_slot = SL_U;
  const T* src = static_cast<const T*>(pd.buf[src_slot]);
  // weights in the order the windows consume them: the forward stencil runs
  // over the reversed PSF
  if (sep) {
    const T* hy = static_cast<const T*>(pd.hy);
    const T* hx = static_cast<const T*>(pd.hx);
    for (int k = tid; k < p; k += NT) {
      s_w[k] = CORR ? hx[k] : hx[p - 1 - k];
      s_w[p + k] = CORR ? hy[k] : hy[p - 1 - k];
    }
  } else {
    // the weights are stored in both orders: one flat, coalesced copy
    const T* tw = static_cast<const T*>(pd.tap_w) + (CORR ? 0 : pd.nrw);
    for (int k = tid; k < pd.nruns; k += NT) s_runs[k] = pd.tap_runs[k];
    for (int k = tid; k < pd.nrw; k += NT) s_w[k] = tw[k];
  }
  // input region
  const int oy0 = ZPAD ? ty0 - 2 * c : ty0 - c;
  const int ox0 = ZPAD ? tx0 - 2 * c : tx0 - c;
  // asynchronous copies straight into shared memory (no registers held, all
  // of a thread's copies in flight together); positions outside the source
  // are zero-filled by a copy of 0 source bytes.  One warp per row, lanes
  // along the row (RX <= 64 + MLBA_MAX_P - 1 = 128: four column passes at
  // most); the row's source index is mapped once.
  // When the tile's columns lie inside the source, every tile row is one
  // contiguous source run: it is copied in 16-byte (or 8-byte) chunks from a
  // chunk-aligned start, the tile sitting xs elements into its shared-memory
  // row (xs = the start's offset from the chunk boundary; the same for every
  // row when the source pitch is a multiple of the chunk); bytes past the
  // source row are zero-filled.  Other tiles map every element.
  int xs = 0;
  {
    const int lane = tid & 31;
    const int pitch = (!ZPAD && pd.bc == BC_RECT) ? pd.nf : n;
    const int sx0 = (!ZPAD && pd.bc == BC_RECT) ? ox0 + c : ox0;
    const bool colin = sx0 >= 0 && sx0 + RX <= pitch;
    // antireflective BCs: outside the image a value is a combination of up to
    // four pixels (Section 2.2), so tiles that reach outside take the
    // per-element path below
    const bool ar = !ZPAD && pd.bc == BC_AR;
    const bool ar_out = ar && !(colin && oy0 >= 0 && oy0 + RY <= n);
    // chunk in elements: 16 bytes when the pitch keeps the rows aligned alike,
    // 8 bytes (FP32) for an even pitch, 0: element by element
    const int c16 = 16 / (int)sizeof(T);
    const int ce = !colin ? 0 : (pitch % c16 == 0 ? c16 : (sizeof(T) == 4 && pitch % 2 == 0 ? 2 : 0));
    if (ar_out) {
      // 1-D antireflection of an extended index: up to two (index, weight)
      // terms; 0 terms past the reach of any output of the image
      auto ar_terms = [&](int e, int (&ix)[2], T (&wt)[2]) -> int {
        if (e >= 0 && e < n) { ix[0] = e; wt[0] = T(1); return 1; }
        const int k = e < 0 ? -e : e - (n - 1);          // distance outside the edge
        if (k > n - 1) return 0;
        ix[0] = e < 0 ? 0 : n - 1;
        ix[1] = e < 0 ? k : n - 1 - k;
        wt[0] = T(2); wt[1] = T(-1);
        return 2;
      };
      for (int idx = tid; idx < RY * RX; idx += NT) {
        const int ry = idx / RX, rx = idx - ry * RX;
        int iy[2], ix[2];
        T wy[2], wx[2];
        const int ny = ar_terms(oy0 + ry, iy, wy), nx = ar_terms(ox0 + rx, ix, wx);
        T v = T(0);
        for (int a = 0; a < ny; ++a)
          for (int b = 0; b < nx; ++b) v += wy[a] * wx[b] * src[(size_t)iy[a] * n + ix[b]];
        s_in[ry * RP + rx] = v;
      }
    } else if (ce > 0) {
      xs = sx0 % ce;
      const int gs = sx0 - xs;
      const int nch = (xs + RX + ce - 1) / ce;      // <= 65 (8-byte chunks of <= 129 values): three passes
      for (int ry = tid >> 5; ry < RY; ry += NT / 32) {
        const int ey = oy0 + ry;
        int sy;
        if (ZPAD) sy = (ey >= 0 && ey < n) ? ey : -1;
        else if (pd.bc == BC_RECT) sy = (ey + c >= 0 && ey + c < pd.nf) ? ey + c : -1;
        else sy = bc_map_near(ey, n, pd.bc);
        const T* row = src + (size_t)(sy < 0 ? 0 : sy) * pitch;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int ch = lane + 32 * k;
          if (ch < nch) {
            const int g0 = gs + ch * ce;
            int nv = pitch - g0;
            nv = nv < 0 ? 0 : (nv > ce ? ce : nv);
            if (sy < 0) nv = 0;
            T* d = s_in + ry * RP + ch * ce;
            const T* g = row + (nv > 0 ? g0 : 0);
            if (ce * (int)sizeof(T) == 16) cp_async_bytes<16>(d, g, nv * (int)sizeof(T));
            else cp_async_bytes<8>(d, g, nv * (int)sizeof(T));
          }
        }
      }
    } else {
      for (int ry = tid >> 5; ry < RY; ry += NT / 32) {
        const int ey = oy0 + ry;
        int sy;
        if (ZPAD) sy = (ey >= 0 && ey < n) ? ey : -1;
        else if (pd.bc == BC_RECT) sy = (ey + c >= 0 && ey + c < pd.nf) ? ey + c : -1;
        else sy = bc_map_near(ey, n, pd.bc);
        const T* row = src + (size_t)(sy < 0 ? 0 : sy) * pitch;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int rx = lane + 32 * k;
          if (rx < RX) {
            const int ex = ox0 + rx;
            int sx;
            if (ZPAD) sx = (ex >= 0 && ex < n) ? ex : -1;
            else if (pd.bc == BC_RECT) sx = (ex + c >= 0 && ex + c < pd.nf) ? ex + c : -1;
            else sx = bc_map_near(ex, n, pd.bc);
            const bool ok = sy >= 0 && sx >= 0;
            cp_async_zfill<sizeof(T)>(s_in + ry * RP + rx, row + (ok ? sx : 0), ok);
          }
        }
      }
    }
    cp_async_wait_all();
  }
  blk.sync();
  // this thread's outputs: columns x2, x2 + 1, rows y8 .. y8 + 7 of the tile
  const int x2 = 2 * (tid & 31), y8 = (tid >> 5) * 8;
  T2 acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) { acc[j].x = T(0); acc[j].y = T(0); }
  if (sep && 8 * RY <= ST_ROW_ITEMS * NT) {
    // row pass over all RY rows, tmp(ry, xx) = sum_t wx[t] in(ry, xx + t): every
    // thread first holds all of its (row, 8 columns) items in registers, then,
    // after a barrier, writes them over the input tile (row ry of tmp at the
    // start of input row ry), so no second tile is needed
    T h[ST_ROW_ITEMS][8];
#pragma unroll
    for (int i = 0; i < ST_ROW_ITEMS; ++i) {
      const int idx = tid + i * NT;
#pragma unroll
      for (int j = 0; j < 8; ++j) h[i][j] = T(0);
      if (idx < 8 * RY) window_run<T>(h[i], s_in + (idx >> 3) * RP + xs + (idx & 7) * 8, 1, s_w, p);
    }
    blk.sync();
#pragma unroll
    for (int i = 0; i < ST_ROW_ITEMS; ++i) {
      const int idx = tid + i * NT;
      if (idx < 8 * RY) {
#pragma unroll
        for (int j = 0; j < 8; ++j) s_in[(idx >> 3) * RP + (idx & 7) * 8 + j] = h[i][j];
      }
    }
    blk.sync();
    // column pass: out(y, x) = sum_t wy[t] tmp(y + t, x)
    window_run2<T>(acc, s_in + y8 * RP + x2, RP, s_w + p, p, true);
  } else if (sep) {
    // (taller tiles, p > 33) the row pass into a second tile
    for (int idx = tid; idx < 8 * RY; idx += NT) {
      const int ry = idx >> 3, x8 = (idx & 7) * 8;
      T h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = T(0);
      window_run<T>(h, s_in + ry * RP + xs + x8, 1, s_w, p);
#pragma unroll
      for (int j = 0; j < 8; ++j) s_tmp[ry * ST_TP + x8 + j] = h[j];
    }
    blk.sync();
    // column pass: out(y, x) = sum_t wy[t] tmp(y + t, x)
    window_run2<T>(acc, s_tmp + y8 * ST_TP + x2, ST_TP, s_w + p, p, true);
  } else {
    // runs of PSF column b over rows lo..hi: input columns x + (CORR ? b : 2c - b),
    // window rows from y8 + (CORR ? lo : 2c - hi)
    for (int k = 0; k < pd.nruns; ++k) {
      const int4 rn = s_runs[k];
      const int len = rn.z - rn.y + 1;
      const int col = CORR ? x2 + rn.x : x2 + 2 * c - rn.x;
      const int r0 = CORR ? y8 + rn.y : y8 + 2 * c - rn.z;
      window_run2<T>(acc, s_in + r0 * RP + xs + col, RP, s_w + rn.w, len, ((xs + col) & 1) == 0);
    }
  }
  T* dst = static_cast<T*>(pd.buf[dst_slot]);
  const T* aux = static_cast<const T*>(pd.buf[aux_slot]);
  T lacc = T(0);
  const int gx = tx0 + x2;
  auto emit = [&](size_t o, T a, T xv) {
    if (MODE == ST_FWD_RESID) {
      const T r = xv - a;
      dst[o] = r;
      lacc += r * r;
    } else if (MODE == ST_FWD_PCGQ) {
      const T pv = xv;
      const T qv = a + T(pd.alpha) * pv;
      dst[o] = qv;
      lacc += pv * qv;
    } else {
      dst[o] = a;
    }
  };
  // the second operand (g or p) for all 16 outputs first, then the stores
  T2 av[8];
  if (MODE == ST_FWD_RESID || MODE == ST_FWD_PCGQ) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gy = ty0 + y8 + j;
      const size_t o = (size_t)gy * outN + gx;
      av[j].x = (gy < outN && gx < outN) ? aux[o] : T(0);
      av[j].y = (gy < outN && gx + 1 < outN) ? aux[o + 1] : T(0);
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int gy = ty0 + y8 + j;
    if (gy < outN) {
      const size_t o = (size_t)gy * outN + gx;
      if (gx < outN) emit(o, acc[j].x, av[j].x);
      if (gx + 1 < outN) emit(o + 1, acc[j].y, av[j].y);
    }
  }
  if (MODE == ST_FWD_RESID || MODE == ST_FWD_PCGQ) {
    // each thread's 16 terms in T; from the warp sum on, FP64 (an FP32
    // partial of 16 squares is within 16 u = 1e-6 of its exact value)
    double dl = (double)lacc;
    for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
    if ((tid & 31) == 0) red[tid >> 5] = dl;
    blk.sync();
    double vals[1] = {0.0};
    if (tid == 0)
      for (int w = 0; w < NT / 32; ++w) vals[0] += red[w];
    blk.sync();
    double tot[1];
    if (last_block_reduce_b<NT, 1>(pd, st, item.y, pd.nblk_blur, vals, tot, red, flag, blk)) {
      if (tid == 0) {
        if (MODE == ST_FWD_RESID) {
          finalize_residual(pd, st, tot[0]);
        } else {
          st.pa = (tot[0] != 0.0) ? st.prho / tot[0] : 0.0;
        }
      }
    }
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(STENCIL_THREADS, sizeof(T) == 4 ? 8 : 4)
k_stencil(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
          int src_slot, int dst_slot, int aux_slot, int pcg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ int flag;
  stencil_body<T, MODE>(items[blockIdx.x], probs, states, src_slot, dst_slot, aux_slot, pcg, smraw,
                        red, &flag, BlkFull{});
}

template <typename T, int MODE>
__global__ void __launch_bounds__(VEC_THREADS)
k_vec(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
      int pcg) {
  __shared__ double red[32];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (st.stopped) return;
  // INIT re-arms the PCG; FINISH always copies the solution out
  if (pcg && st.pdone && MODE != VEC_PCG_INIT && MODE != VEC_PCG_FINISH) return;
  if (MODE == VEC_PCG_INIT && item.y == 0 && threadIdx.x == 0) st.pdone = 0;
  const int n = pd.n;
  const size_t nn = (size_t)n * n;
  const size_t chunk = (size_t)VEC_THREADS * VEC_PER_THREAD;
  const size_t beg = (size_t)item.y * chunk;
  const size_t end = beg + chunk < nn ? beg + chunk : nn;
  T* U = static_cast<T*>(pd.buf[SL_U]);
  T* PX = static_cast<T*>(pd.buf[SL_PX]);
  T* PRES = static_cast<T*>(pd.buf[SL_PRES]);
  T* PP = static_cast<T*>(pd.buf[SL_PP]);
  T* PQ = static_cast<T*>(pd.buf[SL_PQ]);
  T* PZ = static_cast<T*>(pd.buf[SL_PZ]);
  double lacc = 0.0;
  T tacc = T(0);
  for (size_t i = beg + threadIdx.x; i < end; i += VEC_THREADS) {
    if (MODE == VEC_FOLD) {
      const int a = (int)(i / n), b = (int)(i - (size_t)a * n);
      U[i] = fold_fetch<T>(pd, static_cast<const T*>(pd.buf[SL_V]), a, b);
    } else if (MODE == VEC_PCG_INIT) {
      PX[i] = T(0);
      PRES[i] = static_cast<const T*>(pd.buf[SL_R])[i];
    } else if (MODE == VEC_PCG_RHO0) {
      const T zv = PZ[i];
      tacc += PRES[i] * zv;
      PP[i] = zv;
    } else if (MODE == VEC_PCG_AXPY) {
      const T a = T(st.pa);
      PX[i] += a * PP[i];
      PRES[i] -= a * PQ[i];
    } else if (MODE == VEC_PCG_RHO) {
      tacc += PRES[i] * PZ[i];
    } else if (MODE == VEC_PCG_PUPD) {
      PP[i] = PZ[i] + T(st.pbeta) * PP[i];
    } else if (MODE == VEC_PCG_FINISH) {
      static_cast<T*>(pd.buf[SL_T])[i] = PX[i];
    }
  }
  if (MODE == VEC_PCG_RHO0 || MODE == VEC_PCG_RHO) {
    lacc = (double)tacc;
    const double bs = block_sum<VEC_THREADS>(lacc, red);
    double tot[1];
    const double vals[1] = {bs};
    if (last_block_reduce<VEC_THREADS, 1>(pd, st, item.y, pd.nblk_vec, vals, tot, red) &&
        threadIdx.x == 0) {
      const double rho = tot[0];
      if (MODE == VEC_PCG_RHO0) {
        st.prho = rho;
        st.prho0 = rho;
        st.psteps = 0;
        st.pdone = (rho <= 0.0) ? 1 : 0;
      } else {
        st.psteps += 1;
        // relative residual of the symmetric system (psys): sqrt(r_k^T M r_k / r_0^T M r_0)
        const double rel = sqrt(fmax(rho, 0.0) / st.prho0);
        if (rel <= pd.pcg_tol || st.psteps >= pd.pcg_max) {
          st.pdone = 1;
        } else {
          st.pbeta = rho / st.prho;
          st.prho = rho;
        }
      }
    }
  }
  if (MODE == VEC_PCG_FINISH && item.y == 0 && threadIdx.x == 0) {
    const int it = st.iter - 1;
    st.beta_last = st.psteps;
    if (it >= 0 && it < pd.max_iter + 2) pd.hist_beta[it] = st.psteps;
  }
}


// ---------------------------------------------------------------------------
// Blur by FFT convolution (Section 2.1 and 2.2: A and A^T applied with FFTs
// after padding).  Each problem on this path has two convolution entries in
// the problem table, forward and adjoint, of size M >= m = n + p - 1 (their
// `sidx` is the problem), whose spectra are conj(H^) and H^ (H^ = DFT of the
// PSF centred at the origin) with |lambda|^2 = 0, so that the spectral
// column pass with alpha = 1 and the Algorithm-4 weight conj(lambda)/M^2
// multiplies by H^/M^2 (convolution) or conj(H^)/M^2 (correlation).
// Circular convolution of size M >= m has no wrap-around on the samples used:
//   forward:  X = f extended by the BCs (m x m, zero beyond), Y = X (*) h,
//             (A f)(i, j) = Y(i + c, j + c);
//   adjoint:  X = t at offset (c, c), Y = X (x) h, V(a, b) = Y(a, b), a, b < m
//             (antireflective BCs: X = t extended antireflectively,
//             (A' t)(i, j) = Y(i + c, j + c)).

// 1-D antireflection of an extended index into up to two (index, weight) terms
template <typename T>
__device__ __forceinline__ int fc_ar_terms(int e, int n, int (&ix)[2], T (&wt)[2]) {
  if (e >= 0 && e < n) { ix[0] = e; wt[0] = T(1); return 1; }
  const int k = e < 0 ? -e : e - (n - 1);
  if (k > n - 1) return 0;
  ix[0] = e < 0 ? 0 : n - 1;
  ix[1] = e < 0 ? k : n - 1 - k;
  wt[0] = T(2); wt[1] = T(-1);
  return 2;
}

// X of a convolution entry (item.x) from its problem's image: src_slot < 0
// takes f (forward) or t (r for P = I) (adjoint)
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_fc_pad(const Prob* __restrict__ probs, const State* __restrict__ states,
         const int2* __restrict__ items, int adj, int src_slot) {
  const int2 item = items[blockIdx.x];
  const Prob& sh = probs[item.x];
  const Prob& pd = probs[sh.sidx];
  if (states[sh.sidx].stopped) return;
  const int M = sh.n, n = pd.n, c = pd.c, m = pd.ne;
  const size_t MM = (size_t)M * M;
  if (src_slot < 0) src_slot = adj ? (pd.precond == P_NONE ? SL_R : SL_T) : SL_F;
  const T* src = static_cast<const T*>(pd.buf[src_slot]);
  T* X = static_cast<T*>(sh.buf[SL_R]);
  const bool ext = !adj || pd.bc == BC_AR;          // BC-extended input on [0, m)^2
  const size_t beg = (size_t)item.y * VEC_THREADS * VEC_PER_THREAD;
  for (size_t e = beg + threadIdx.x; e < beg + VEC_THREADS * VEC_PER_THREAD && e < MM; e += VEC_THREADS) {
    const int y = (int)(e / M), x = (int)(e - (size_t)y * M);
    T v = T(0);
    if (ext) {
      if (y < m && x < m) {
        if (pd.bc == BC_RECT) {
          v = src[(size_t)y * m + x];
        } else if (pd.bc == BC_AR) {
          int iy[2], ix[2];
          T wy[2], wx[2];
          const int ny = fc_ar_terms<T>(y - c, n, iy, wy), nx = fc_ar_terms<T>(x - c, n, ix, wx);
          for (int a = 0; a < ny; ++a)
            for (int b = 0; b < nx; ++b) v += wy[a] * wx[b] * src[(size_t)iy[a] * n + ix[b]];
        } else {
          const int sy = bc_map(y - c, n, pd.bc), sx = bc_map(x - c, n, pd.bc);
          if (sy >= 0 && sx >= 0) v = src[(size_t)sy * n + sx];
        }
      }
    } else if (y >= c && y < c + n && x >= c && x < c + n) {
      v = src[(size_t)(y - c) * n + (x - c)];
    }
    X[e] = v;
  }
}

// from the convolution entry's Y to the problem (item.x = problem):
//   FC_RESID: r = g - Y(i + c, j + c), ||r||^2 and the stop rule (as the
//             residual stencil), FC_STORE: dst = Y(i + c, j + c) (n x n),
//   FC_CORR: V = Y on [0, m)^2
enum { FC_RESID = 0, FC_STORE = 1, FC_CORR = 2 };
template <typename T, int MODE>
__global__ void __launch_bounds__(VEC_THREADS)
k_fc_out(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
         int adj, int dst_slot) {
  __shared__ double red[32];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (st.stopped) return;
  const Prob& sh = probs[pd.fc_sh[adj]];
  const int M = sh.n, n = pd.n, c = pd.c, m = pd.ne;
  const T* Y = static_cast<const T*>(sh.buf[SL_T]);
  const int w = (MODE == FC_CORR) ? m : n;
  const size_t tot = (size_t)w * w;
  const int off = (MODE == FC_CORR) ? 0 : c;
  T* dst = static_cast<T*>(pd.buf[dst_slot]);
  const T* g = static_cast<const T*>(pd.buf[SL_G]);
  const size_t beg = (size_t)item.y * VEC_THREADS * VEC_PER_THREAD;
  T lacc = T(0);
  for (size_t e = beg + threadIdx.x; e < beg + VEC_THREADS * VEC_PER_THREAD && e < tot; e += VEC_THREADS) {
    const int y = (int)(e / w), x = (int)(e - (size_t)y * w);
    const T yv = Y[(size_t)(y + off) * M + (x + off)];
    if (MODE == FC_RESID) {
      const T r = g[e] - yv;
      dst[e] = r;
      lacc += r * r;
    } else {
      dst[e] = yv;
    }
  }
  if (MODE == FC_RESID) {
    // (each thread's terms in T, FP64 from the block sum on, fixed order)
    const double bs = block_sum<VEC_THREADS>((double)lacc, red);
    const double vals[1] = {bs};
    double tot1[1];
    if (last_block_reduce<VEC_THREADS, 1>(pd, st, item.y, pd.nblk_vec, vals, tot1, red) &&
        threadIdx.x == 0)
      finalize_residual(pd, st, tot1[0]);
  }
}

// Balanced formulation: the framelet step's input becomes f + u, with u as
// the step left it: the BC fold of V (written to U), V (rectangular A, in
// place), U (A' t of antireflective BCs, in place) or t (Algorithm 4 forms,
// in place).  item.y: block of the N_f^2 plane.
template <typename T>
__device__ __forceinline__ void balance_body(const int2 item, const Prob* __restrict__ probs,
                                             const State* __restrict__ states) {
  const Prob& pd = probs[item.x];
  if (states[item.x].stopped) return;
  const int nf = pd.nf;
  const size_t tot = (size_t)nf * nf;
  const T* F = static_cast<const T*>(pd.buf[SL_F]);
  const bool fold = pd.use_adj && pd.bc != BC_RECT && pd.bc != BC_AR;
  T* dst = static_cast<T*>(pd.buf[!pd.use_adj ? SL_T : (pd.bc == BC_RECT ? SL_V : SL_U)]);
  const T* V = static_cast<const T*>(pd.buf[SL_V]);
  const size_t beg = (size_t)item.y * VEC_THREADS * VEC_PER_THREAD;
  for (size_t e = beg + threadIdx.x; e < beg + VEC_THREADS * VEC_PER_THREAD && e < tot; e += VEC_THREADS) {
    const int a = (int)(e / nf), b = (int)(e - (size_t)a * nf);
    const T u = fold ? fold_fetch<T>(pd, V, a, b) : dst[e];
    dst[e] = F[e] + u;
  }
}
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS)
k_balance(const Prob* __restrict__ probs, const State* __restrict__ states,
          const int2* __restrict__ items) {
  balance_body<T>(items[blockIdx.x], probs, states);
}

#ifndef MLBA_BODIES_ONLY  // launchers: not in the persistent kernel's unit
template <typename T>
void launch_balance(const Prob* probs, State* states, const int2* items, int nitems, cudaStream_t s) {
  if (nitems > 0) k_balance<T><<<nitems, VEC_THREADS, 0, s>>>(probs, states, items);
}

template <typename T>
void launch_fc_pad(const Prob* probs, State* states, const int2* items, int nitems, int adj,
                   int src_slot, cudaStream_t s) {
  if (nitems > 0) k_fc_pad<T><<<nitems, VEC_THREADS, 0, s>>>(probs, states, items, adj, src_slot);
}
template <typename T>
void launch_fc_out(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                   int adj, int dst_slot, cudaStream_t s) {
  if (nitems <= 0) return;
  if (mode == FC_RESID) k_fc_out<T, FC_RESID><<<nitems, VEC_THREADS, 0, s>>>(probs, states, items, adj, dst_slot);
  else if (mode == FC_STORE) k_fc_out<T, FC_STORE><<<nitems, VEC_THREADS, 0, s>>>(probs, states, items, adj, dst_slot);
  else k_fc_out<T, FC_CORR><<<nitems, VEC_THREADS, 0, s>>>(probs, states, items, adj, dst_slot);
}

// ---------------------------------------------------------------------------
template <typename T>
void launch_stencil(int mode, const Prob* probs, State* states, const int2* items, int nitems,
                    int src, int dst, int aux, int pcg, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return;
  dim3 g(nitems), b(STENCIL_THREADS);
  switch (mode) {
    case ST_FWD_RESID: k_stencil<T, ST_FWD_RESID><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    case ST_FWD_STORE: k_stencil<T, ST_FWD_STORE><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    case ST_FWD_PCGQ: k_stencil<T, ST_FWD_PCGQ><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    case ST_REBLUR: k_stencil<T, ST_REBLUR><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    default: k_stencil<T, ST_CORR><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
  }
}

template <typename T>
cudaError_t stencil_set_smem(size_t bytes) {
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_stencil<T, ST_FWD_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_stencil<T, ST_FWD_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_stencil<T, ST_FWD_PCGQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_stencil<T, ST_REBLUR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stencil<T, ST_CORR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
void launch_vec(int mode, const Prob* probs, State* states, const int2* items, int nitems,
                int pcg, cudaStream_t s) {
  if (nitems <= 0) return;
  dim3 g(nitems), b(VEC_THREADS);
  switch (mode) {
    case VEC_FOLD: k_vec<T, VEC_FOLD><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    case VEC_PCG_INIT: k_vec<T, VEC_PCG_INIT><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    case VEC_PCG_RHO0: k_vec<T, VEC_PCG_RHO0><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    case VEC_PCG_AXPY: k_vec<T, VEC_PCG_AXPY><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    case VEC_PCG_RHO: k_vec<T, VEC_PCG_RHO><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    case VEC_PCG_PUPD: k_vec<T, VEC_PCG_PUPD><<<g, b, 0, s>>>(probs, states, items, pcg); break;
    default: k_vec<T, VEC_PCG_FINISH><<<g, b, 0, s>>>(probs, states, items, pcg); break;
  }
}

template void launch_stencil<float>(int, const Prob*, State*, const int2*, int, int, int, int, int, size_t, cudaStream_t);
template void launch_stencil<double>(int, const Prob*, State*, const int2*, int, int, int, int, int, size_t, cudaStream_t);
template cudaError_t stencil_set_smem<float>(size_t);
template cudaError_t stencil_set_smem<double>(size_t);
template void launch_balance<float>(const Prob*, State*, const int2*, int, cudaStream_t);
template void launch_balance<double>(const Prob*, State*, const int2*, int, cudaStream_t);
template void launch_fc_pad<float>(const Prob*, State*, const int2*, int, int, int, cudaStream_t);
template void launch_fc_pad<double>(const Prob*, State*, const int2*, int, int, int, cudaStream_t);
template void launch_fc_out<float>(const Prob*, State*, const int2*, int, int, int, int, cudaStream_t);
template void launch_fc_out<double>(const Prob*, State*, const int2*, int, int, int, int, cudaStream_t);
template void launch_vec<float>(int, const Prob*, State*, const int2*, int, int, cudaStream_t);
template void launch_vec<double>(int, const Prob*, State*, const int2*, int, int, cudaStream_t);

#endif  // MLBA_BODIES_ONLY

}  // namespace mlba
