// k_frame.cu — fused undecimated B-spline framelet step of Eq. MLBA2:
//
//     z_out = z_in + W u,   x = S_mu(z_out),   f = W^T x
//
// W is the L-level undecimated transform of Section 6.1 (masks b0, b1, b2,
// dilated by 2^(l-1) at level l, half-sample reflective boundary).  One CTA
// owns a 32 x 32 tile of f and of every z band.  Everything is computed on
// the reflectively extended domain around the tile: u is loaded with a halo
// of 2(2^L - 1) pixels, z with the halo each band needs (2^l - 1), taking
// z outside the image from its mirror image with the sign of the band's
// symmetry (b1 is antisymmetric).  The extension of W u under the same
// mirroring equals W of the extended u, and S_mu is odd, so every value on
// the halo is exact and W^T reduces to plain (dilated) convolutions there.
// z is read once per band from a ping-pong buffer (no in-place race between
// neighbouring tiles) and written once for the tile interior.
//
// u comes from (per problem): the full correlation V folded by the BC
// transpose (A^T t for imposed boundary conditions), V itself (rectangular
// A), or t (Algorithm 4 forms, where C^T is already applied).
#include "mlba_internal.cuh"
#include "mlba_launch.h"

namespace mlba {

__device__ __constant__ float c_mask_f[3][3] = {
    {0.25f, 0.5f, 0.25f},
    {0.35355339059327376220f, 0.0f, -0.35355339059327376220f},
    {-0.25f, 0.5f, -0.25f}};
__device__ __constant__ double c_mask_d[3][3] = {
    {0.25, 0.5, 0.25},
    {0.35355339059327376220, 0.0, -0.35355339059327376220},
    {-0.25, 0.5, -0.25}};

template <typename T> __device__ __forceinline__ T mask(int k, int t);
template <> __device__ __forceinline__ float mask<float>(int k, int t) { return c_mask_f[k][t]; }
template <> __device__ __forceinline__ double mask<double>(int k, int t) { return c_mask_d[k][t]; }

template <typename T> __device__ __forceinline__ T soft_thr(T v, T mu) {
  const T a = fabs(v) - mu;
  return a > T(0) ? copysign(a, v) : T(0);
}

__host__ __device__ __forceinline__ int xr(int l) { return (1 << l) - 1; }   // X_l = 2^l - 1
// radius of the level-l low-pass c_l that the tile needs: X_L + 2^L - 2^l
__host__ __device__ __forceinline__ int cr(int l, int L) { return xr(L) + (1 << L) - (1 << l); }

template <typename T, typename TZ>
size_t frame_smem_bytes(int L) {
  const int TS = FRAME_TILE;
  size_t e = 0;
  const int w0 = TS + 2 * cr(0, L), w1 = TS + 2 * cr(L > 1 ? 1 : 0, L);
  e += (size_t)w0 * w0 + (size_t)w1 * w1;               // c ping-pong
  e += (size_t)(TS + 2 * xr(L)) * (TS + 2 * xr(L));     // one x band
  for (int l = 0; l < L; ++l) e += (size_t)(TS + 2 * xr(l)) * (TS + 2 * xr(l));   // s_l
  return e * sizeof(T);
}

template <typename T, typename TZ>
__global__ void __launch_bounds__(FRAME_THREADS)
k_frame(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
        int u_slot, int f_slot, const void* zin_op, void* zout_op, double op_mu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  const State& st = states[item.x];
  if (st.stopped) return;
  const int TS = FRAME_TILE;
  const int L = pd.levels, nf = pd.nf;
  const int tilesX = (nf + TS - 1) / TS;
  const int by0 = (item.y / tilesX) * TS, bx0 = (item.y % tilesX) * TS;
  const T mu = T(zin_op ? op_mu : pd.mu);
  const TZ* zin;
  TZ* zout;
  if (zin_op) {
    zin = static_cast<const TZ*>(zin_op);
    zout = static_cast<TZ*>(zout_op);
  } else {
    zin = static_cast<const TZ*>(pd.z[(st.iter - 1) & 1]);
    zout = static_cast<TZ*>(pd.z[st.iter & 1]);
  }
  const size_t plane = (size_t)nf * nf;

  // shared memory carve-up
  T* cA = reinterpret_cast<T*>(smraw);
  const int w0 = TS + 2 * cr(0, L);
  T* cB = cA + w0 * w0;
  const int w1 = TS + 2 * cr(L > 1 ? 1 : 0, L);
  T* xb = cB + w1 * w1;
  const int wx = TS + 2 * xr(L);
  T* sbuf[MAX_LEVELS];
  {
    T* q = xb + wx * wx;
    for (int l = 0; l < L; ++l) { sbuf[l] = q; q += (TS + 2 * xr(l)) * (TS + 2 * xr(l)); }
  }

  // 1. u on the extended tile (radius C_0 = 2(2^L - 1))
  {
    const int C0 = cr(0, L);
    int mode;          // 0: V folded, 1: direct nf x nf array
    const T* src;
    if (u_slot >= 0) { src = static_cast<const T*>(pd.buf[u_slot]); mode = 1; }
    else if (!pd.use_adj) { src = static_cast<const T*>(pd.buf[SL_T]); mode = 1; }
    else if (pd.bc == BC_RECT) { src = static_cast<const T*>(pd.buf[SL_V]); mode = 1; }
    else { src = static_cast<const T*>(pd.buf[SL_V]); mode = 0; }
    for (int idx = threadIdx.x; idx < w0 * w0; idx += FRAME_THREADS) {
      const int ry = idx / w0, rx = idx - ry * w0;
      int o;
      const int ay = refl_half(by0 - C0 + ry, nf, &o);
      const int ax = refl_half(bx0 - C0 + rx, nf, &o);
      cA[idx] = mode ? src[(size_t)ay * nf + ax] : fold_fetch<T>(pd, src, ay, ax);
    }
  }
  // zero the synthesis accumulators
  for (int l = 0; l < L; ++l) {
    const int ws = TS + 2 * xr(l);
    for (int idx = threadIdx.x; idx < ws * ws; idx += FRAME_THREADS) sbuf[l][idx] = T(0);
  }
  __syncthreads();

  // 2. levels, bottom-up: analysis, update, threshold, synthesis of the bands
  T* cur = cA;
  T* nxt = cB;
  int wc = w0, rc = cr(0, L);
  for (int lev = 1; lev <= L; ++lev) {
    const int D = 1 << (lev - 1);
    const int X = xr(lev), wxl = TS + 2 * X;
    const int Xs = xr(lev - 1), ws = TS + 2 * Xs;
    T* s = sbuf[lev - 1];
    const int nb = (lev == L) ? 9 : 8;
    for (int b = 0; b < nb; ++b) {
      int bi, bj;
      if (b == 8) { bi = 0; bj = 0; } else { const int q = b + 1; bi = q / 3; bj = q % 3; }
      const int band = (b == 8) ? 8 * L : (lev - 1) * 8 + b;
      const TZ* zi = zin + band * plane;
      TZ* zo = zout + band * plane;
      const int off = rc - X;   // offset of the band region inside cur
      // a. analysis + update + threshold on radius X
      for (int idx = threadIdx.x; idx < wxl * wxl; idx += FRAME_THREADS) {
        const int qy = idx / wxl, qx = idx - qy * wxl;
        T val = T(0);
#pragma unroll
        for (int sy = 0; sy < 3; ++sy) {
          const T my = mask<T>(bi, sy);
          if (my == T(0)) continue;
          T rowacc = T(0);
          const T* crow = cur + (qy + off + (sy - 1) * D) * wc + qx + off;
#pragma unroll
          for (int sx = 0; sx < 3; ++sx) {
            const T mx = mask<T>(bj, sx);
            if (mx != T(0)) rowacc += mx * crow[(sx - 1) * D];
          }
          val += my * rowacc;
        }
        const int gy = by0 - X + qy, gx = bx0 - X + qx;
        int oy, ox;
        const int zy = refl_half(gy, nf, &oy), zx = refl_half(gx, nf, &ox);
        const bool neg = ((bi == 1) && oy) != ((bj == 1) && ox);
        T zo_v = T(ld_z(zi + (size_t)zy * nf + zx));
        if (neg) zo_v = -zo_v;
        const T zn = zo_v + val;
        if (qy >= X && qy < X + TS && qx >= X && qx < X + TS && gy < nf && gx < nf)
          st_z(zo + (size_t)gy * nf + gx, zn);
        xb[idx] = soft_thr<T>(zn, mu);
      }
      __syncthreads();
      // b. synthesis of this band into s_{lev-1} on radius Xs (convolution)
      for (int idx = threadIdx.x; idx < ws * ws; idx += FRAME_THREADS) {
        const int qy = idx / ws, qx = idx - qy * ws;
        T acc = T(0);
#pragma unroll
        for (int sy = 0; sy < 3; ++sy) {
          const T my = mask<T>(bi, sy);
          if (my == T(0)) continue;
          T rowacc = T(0);
          const T* xrow = xb + (qy + D - (sy - 1) * D) * wxl + qx + D;
#pragma unroll
          for (int sx = 0; sx < 3; ++sx) {
            const T mx = mask<T>(bj, sx);
            if (mx != T(0)) rowacc += mx * xrow[-(sx - 1) * D];
          }
          acc += my * rowacc;
        }
        s[idx] += acc;
      }
      __syncthreads();
    }
    if (lev < L) {
      // next low-pass c_lev on its radius
      const int rn = cr(lev, L), wn = TS + 2 * rn;
      const int off = rc - rn;
      for (int idx = threadIdx.x; idx < wn * wn; idx += FRAME_THREADS) {
        const int qy = idx / wn, qx = idx - qy * wn;
        T val = T(0);
#pragma unroll
        for (int sy = 0; sy < 3; ++sy) {
          T rowacc = T(0);
          const T* crow = cur + (qy + off + (sy - 1) * D) * wc + qx + off;
#pragma unroll
          for (int sx = 0; sx < 3; ++sx) rowacc += mask<T>(0, sx) * crow[(sx - 1) * D];
          val += mask<T>(0, sy) * rowacc;
        }
        nxt[idx] = val;
      }
      __syncthreads();
      T* tmp = cur; cur = nxt; nxt = tmp;
      wc = wn; rc = rn;
    }
  }
  // 3. top-down: s_{l-1} += (b0 x b0, dilation 2^(l-1)) * s_l
  for (int lev = L - 1; lev >= 1; --lev) {
    const int D = 1 << (lev - 1);
    const int wl = TS + 2 * xr(lev), ws = TS + 2 * xr(lev - 1);
    const T* sl = sbuf[lev];
    T* sd = sbuf[lev - 1];
    for (int idx = threadIdx.x; idx < ws * ws; idx += FRAME_THREADS) {
      const int qy = idx / ws, qx = idx - qy * ws;
      T acc = T(0);
#pragma unroll
      for (int sy = 0; sy < 3; ++sy) {
        T rowacc = T(0);
        const T* row = sl + (qy + D - (sy - 1) * D) * wl + qx + D;
#pragma unroll
        for (int sx = 0; sx < 3; ++sx) rowacc += mask<T>(0, sx) * row[-(sx - 1) * D];
        acc += mask<T>(0, sy) * rowacc;
      }
      sd[idx] += acc;
    }
    __syncthreads();
  }
  // 4. f = s_0 on the tile
  T* f = static_cast<T*>(pd.buf[f_slot]);
  for (int idx = threadIdx.x; idx < TS * TS; idx += FRAME_THREADS) {
    const int qy = idx / TS, qx = idx - qy * TS;
    const int gy = by0 + qy, gx = bx0 + qx;
    if (gy < nf && gx < nf) f[(size_t)gy * nf + gx] = sbuf[0][idx];
  }
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (one thread, 4 or 8 bytes) and their groups
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) for the z rows of the ring variant of the framelet sweep.  Every
// wait on an mbarrier is bounded: after about one second (global timer) or
// Z_SPIN_LIMIT polls it gives up and the caller reports MLBA_E_TIMEOUT
// instead of hanging.
constexpr unsigned Z_SPIN_LIMIT = 1u << 26;
constexpr unsigned long long Z_WAIT_NS = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// true once the phase with the given parity has completed; false after the
// spin limit
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  const unsigned a = smem_u32(b);
  unsigned long long t0 = 0;
  for (unsigned it = 0; it < Z_SPIN_LIMIT; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = global_ns();
    else if ((it & 255) == 0 && global_ns() - t0 > Z_WAIT_NS) return false;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Warp row-sweep variant for L <= 2 (the measured workloads).
//
// A CTA owns an F3_TX x (32 F3_NWR) tile of f and of every z band; warp w
// owns the 32-row segment w of it.  In each level a lane owns one column of
// the band region (coefficients at columns tx0 - X .. tx0 - X + 31) and the
// warp sweeps down the rows:
//   analysis   h_j(y, x) = sum_t b_j[t] c(y, x + (t-1)D)     (shared memory)
//              a_ij(y, x) = sum_s b_i[s] h_j(y + (s-1)D, x)  (register ring)
//   update     z' = z + a, x_ij = S_mu(z')                   (z in registers,
//              loaded PF rows ahead straight from global memory)
//   synthesis  P_j(y + (s-1)D) += b_i[s] x_ij                (register ring)
//              out(y, x) = A(x + D) + B(x) + C(x - D)         (warp shuffles)
//              with A, B, C = sum_j b_j[0], b_j[1], b_j[2] P_j
// Every lane computes a coefficient column, but only lanes whose +-D
// neighbours are in the warp produce output: level 2 (D = 2) lanes 2..29,
// level 1 lanes 1..26.  Neighbouring warps and tiles recompute the
// overlapping coefficients (from the same z_in) and only the owner writes
// z_out.  Shared memory carries only the input u (c_1 = (b0 x b0) u is formed
// on the fly by the level-2 sweep) and the level-2 part of f, so there are no
// shared-memory atomics; the only CTA-wide barrier follows the u tile.
constexpr int F3_TX = 26;      // tile columns: level-2 output lanes 3..28 after the +-1 low-pass
constexpr int F3_SEG = 32;     // rows per warp
// Tile shapes the autotuner chooses from: warps (32-row segments) per CTA and
// the z prefetch distance in rows.  Every shape computes the same values in
// the same order (a warp's sweep does not depend on its CTA), so the choice
// changes the time only.  Shape 0 is the default; FP64 always uses it.
// Shapes with ring > 0 stream each warp's z rows through a ring of `ring`
// row slots in shared memory, filled by bulk asynchronous copies (one 1 KB
// copy per row for FP32 z, 512 B for BF16) so that many rows are in flight
// without holding registers; warps whose 32 columns cross the left or right
// image edge (mirrored columns) fill the same ring with per-lane 16-byte
// asynchronous copies.
struct F3Shape { int nwr, pf, ring; };
constexpr F3Shape F3_SHAPES[FRAME_SHAPES] = {{2, 2, 0}, {1, 2, 0}, {4, 2, 0}, {2, 3, 0}, {1, 3, 0},
                                             {2, 2, 6}, {2, 2, 10}, {1, 2, 12}};

template <int L, int NWR>
struct F3 {
  static constexpr int TY = F3_SEG * NWR;
  static constexpr int C0 = (L == 2) ? 6 : 2;         // radius of the u tile
  static constexpr int UW = F3_TX + 2 * C0, UH = TY + 2 * C0;
  static constexpr size_t elems = (size_t)UW * UH + (L == 2 ? (size_t)F3_TX * TY : 0);
};
// bytes of one ring slot: 32 pixels' groups of 8 z values
template <typename TZ>
__host__ __device__ constexpr size_t f3_slot_bytes() { return 32 * 8 * sizeof(TZ); }
// shared memory: u tile and level-2 part of f (T), then per warp `ring` slots
// and `ring` mbarriers
template <typename T, typename TZ, int L, int NWR, int RING>
__host__ __device__ constexpr size_t frame3_ring_offset() {
  return (F3<L, NWR>::elems * sizeof(T) + 15) / 16 * 16;
}
template <typename T, typename TZ, int L, int NWR, int RING>
__host__ __device__ constexpr size_t frame3_smem_bytes() {
  return frame3_ring_offset<T, TZ, L, NWR, RING>() + (size_t)NWR * RING * (f3_slot_bytes<TZ>() + 8);
}

// half-sample reflection of an index with the parity of the mirroring; the
// common cases (inside, or one mirror away) avoid the division
__device__ __forceinline__ int f3_refl(int e, int n, bool* par) {
  if (e >= 0 && e < n) { *par = false; return e; }
  if (e < 0 && e >= -n) { *par = true; return -1 - e; }
  if (e >= n && e < 2 * n) { *par = true; return 2 * n - 1 - e; }
  int o;
  const int r = refl_half(e, n, &o);
  *par = o != 0;
  return r;
}

// Grouped z layout (L <= 2): the 8 high-pass bands of level l of pixel q are
// contiguous, at (l - 1) 8 nf^2 + 8 q + (3 i + j - 1); the final low-pass band
// keeps its plane at 8 L nf^2 + q.  A lane then moves one pixel's bands of a
// level with one to four 16-byte accesses and one address.
template <typename TZ>
union ZGroup {
  uint4 v[8 * sizeof(TZ) / 16];
  TZ e[8];
};
__device__ __forceinline__ float to_z(float v, float*) { return v; }
__device__ __forceinline__ double to_z(double v, double*) { return v; }
__device__ __forceinline__ __nv_bfloat16 to_z(float v, __nv_bfloat16*) { return __float2bfloat16_rn(v); }

// A warp's ring of z rows (RING > 0): slot k holds one row's 32 groups at
// buf + k * 256 values and completes on bar[k]; seq counts the rows that went
// through the bulk path (every bulk row advances one slot and, every RING rows,
// the expected parity); bad is set when a bounded wait gave up.
template <typename TZ>
struct F3Ring {
  TZ* buf;
  unsigned long long* bar;
  int seq;
  bool bad;
};

template <typename T, typename TZ, int LEV, int L, int F3_PF, int RING>
__device__ __forceinline__ void f3_level(const Prob& pd, const T* __restrict__ cin, int cpitch,
                                         int cy0, int cx0, const TZ* __restrict__ zin,
                                         TZ* __restrict__ zout, int ty0, int tx0, int seg_lo,
                                         int seg_hi, T mu, T* __restrict__ f2s,
                                         T* __restrict__ fout, F3Ring<TZ>& rg) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int D = 1 << (LEV - 1);
  constexpr bool TOP = (LEV == L);
  constexpr int XO = (LEV == 2) ? 3 : 1;                 // first coefficient column tx0 - XO
  constexpr int NL = (LEV == 2) ? 32 : F3_TX + 2;        // lanes with a coefficient column
  constexpr int K0 = TOP ? 0 : 1;                        // band k = 3 j + i; (0,0) only at level L
  constexpr int NB = 9 - K0;
  const T s2q = T(0.35355339059327376220);               // sqrt(2) / 4
  const int lane = threadIdx.x & 31;
  const int x = tx0 - XO + lane;
  const bool act = lane < NL;
  const int nf = pd.nf;
  const int plane = nf * nf;     // nbands nf^2 < 2^31 is checked at set-up
  // rows: outputs [yo0, yo1), coefficients [yc0, yc1)
  const int yo0 = (LEV == 2) ? seg_lo - 1 : seg_lo;
  const int yo1 = (LEV == 2) ? seg_hi + 1 : seg_hi;
  const int yc0 = yo0 - D, yc1 = yo1 + D;
  // column part of the z offsets and its mirroring parity
  bool pcx;
  const int zc = f3_refl(x, nf, &pcx);
  const T scol = pcx ? T(-1) : T(1);
  const bool own_c = act && x >= tx0 && x < tx0 + F3_TX && x < nf;
  const T* ccol = cin + (act ? x - cx0 : D);   // idle lanes read a valid column
  // level 2 reads c_1 = (b0 x b0) u, formed here from the u tile: lane l keeps
  // c_1 at columns x - 2 and x + 2 (a sliding ring of the horizontally
  // filtered u rows, g), and gets c_1 at x from lane l - 2 (or l + 2)
  const T* ua = cin + (x - 2 - cx0);
  T gr[3][2];
  auto grow = [&](int y, T (&g)[2]) {
    const T* r = ua + (y - cy0) * cpitch;
    g[0] = T(0.25) * (r[-1] + r[1]) + T(0.5) * r[0];
    g[1] = T(0.25) * (r[3] + r[5]) + T(0.5) * r[4];
  };
  // this level's band group and (top level) the low-pass plane
  constexpr int NV = 8 * (int)sizeof(TZ) / 16;
  const int gbase = (LEV - 1) * 8 * plane, lbase = 8 * L * plane;
  // h ring: rows y - D .. y + D of the current coefficient row y
  T hr[2 * D + 1][3];
  auto hrow = [&](int y, T (&h)[3]) {
    T cm, c0, cp;
    if constexpr (LEV == 2) {
      // rows are requested in order: g holds rows y - 1, y and gets y + 1
      grow(y + 1, gr[2]);
      cm = T(0.25) * (gr[0][0] + gr[2][0]) + T(0.5) * gr[1][0];
      cp = T(0.25) * (gr[0][1] + gr[2][1]) + T(0.5) * gr[1][1];
      const T up = __shfl_up_sync(FULL, cp, 2), dn = __shfl_down_sync(FULL, cm, 2);
      c0 = lane >= 2 ? up : dn;
#pragma unroll
      for (int q = 0; q < 2; ++q) { gr[0][q] = gr[1][q]; gr[1][q] = gr[2][q]; }
    } else {
      const T* r = ccol + (y - cy0) * cpitch;
      cm = r[-D]; c0 = r[0]; cp = r[D];
    }
    const T sp = cm + cp;
    h[0] = T(0.25) * sp + T(0.5) * c0;
    h[1] = s2q * (cm - cp);
    h[2] = T(0.5) * c0 - T(0.25) * sp;
  };
  if constexpr (LEV == 2) {
    grow(yc0 - D - 1, gr[0]);
    grow(yc0 - D, gr[1]);
  }
#pragma unroll
  for (int k = 0; k < 2 * D; ++k) hrow(yc0 - D + k, hr[k]);
  // z queue: rows y .. y + PF - 1 (group and low-pass value per row; with a
  // ring, the low-pass value only)
  ZGroup<TZ> zq[RING > 0 ? 1 : F3_PF];
  TZ zl[F3_PF];
  // (idle lanes load a valid mirrored column too; their values are unused.
  // Offsets stay in 32 bits: nbands nf^2 < 2^31.)
  auto zload = [&](int y, int k) {
    bool par;
    const int q = f3_refl(y, nf, &par) * nf + zc;
    if constexpr (RING == 0) {
      const uint4* src = reinterpret_cast<const uint4*>(zin + (gbase + 8 * q));
#pragma unroll
      for (int v = 0; v < NV; ++v) zq[k].v[v] = src[v];
    }
    if (TOP) zl[k] = zin[lbase + q];
  };
#pragma unroll
  for (int k = 0; k < F3_PF; ++k) zload(yc0 + k, k);
  // ring: rows are issued RING ahead of the sweep.  Bulk path when the warp's
  // 32 columns lie inside the image (one contiguous run of 32 groups per row),
  // else per-lane 16-byte asynchronous copies of the mirrored columns.
  const int x0 = tx0 - XO;
  const bool bulk = RING > 0 && x0 >= 0 && x0 + 32 <= nf;
  const int nrows = yc1 - yc0;
  const int seq0 = rg.seq;
  int n_issued = 0, first_bad = nrows;      // bulk rows issued; first row whose wait gave up
  auto issue = [&](int i) {                 // row yc0 + i into its slot
    if constexpr (RING > 0) {
      bool par;
      const int yr = f3_refl(yc0 + i, nf, &par);
      if (bulk) {
        const int slot = (seq0 + i) % RING;
        ++n_issued;
        if (lane == 0) {
          // (the slot's previous row was only read, by this warp, before the
          // __syncwarp that precedes this copy: no proxy fence is needed)
          mbar_expect_tx(rg.bar + slot, (unsigned)f3_slot_bytes<TZ>());
          bulk_g2s(rg.buf + slot * 256, zin + (gbase + 8 * (yr * nf + x0)),
                   (unsigned)f3_slot_bytes<TZ>(), rg.bar + slot);
        }
      } else {
        const int slot = i % RING;
        const TZ* src = zin + (gbase + 8 * (yr * nf + zc));
        TZ* dst = rg.buf + slot * 256 + 8 * lane;
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async_16(dst + v * (16 / (int)sizeof(TZ)), src + v * (16 / (int)sizeof(TZ)));
        cp_commit();
      }
    }
  };
  if constexpr (RING > 0) {
    // the ring may hold rows an earlier level wrote with per-lane copies:
    // order those writes before this level's bulk copies
    if (bulk && lane == 0) fence_proxy_async();
    for (int i = 0; i < RING; ++i) {
      if (i < nrows) issue(i);
      else if (!bulk) cp_commit();          // empty group: one group per row slot
    }
  }
  // synthesis ring: rows y - D .. y + D
  T pr[2 * D + 1][3];
#pragma unroll
  for (int k = 0; k <= 2 * D; ++k) pr[k][0] = pr[k][1] = pr[k][2] = T(0);
  // level-2 low-pass ring of the horizontally filtered s_1 rows r-2, r-1, r
  T gq[3] = {T(0), T(0), T(0)};
  // one coefficient row; queue slot kq holds its z and is refilled with row
  // y + PF.  The queue is indexed statically (the sweep is unrolled by PF) so
  // that no register receiving an outstanding load is copied before it is used.
  auto step = [&](int y, int kq) {
    if constexpr (RING > 0) {
      // this row's groups from the ring, then the slot is refilled with row y + RING
      const int i = y - yc0;
      if (bulk) {
        const int g = seq0 + i;
        if (!rg.bad && !mbar_wait(rg.bar + g % RING, (unsigned)(g / RING) & 1u)) {
          rg.bad = true;
          first_bad = i;
        }
        const uint4* sv = reinterpret_cast<const uint4*>(rg.buf + (g % RING) * 256 + 8 * lane);
#pragma unroll
        for (int v = 0; v < NV; ++v) zq[0].v[v] = sv[v];
      } else {
        cp_wait<RING - 1>();
        const uint4* sv = reinterpret_cast<const uint4*>(rg.buf + (i % RING) * 256 + 8 * lane);
#pragma unroll
        for (int v = 0; v < NV; ++v) zq[0].v[v] = sv[v];
      }
      __syncwarp();
      if (i + RING < nrows && !rg.bad) issue(i + RING);
      else if (!bulk) cp_commit();
    }
    hrow(y + D, hr[2 * D]);
    bool pry;
    const int zro = f3_refl(y, nf, &pry) * nf;
    // z outside the image is its mirror image; antisymmetric (b1) bands
    // change sign under an odd number of mirrorings
    const T srow = pry ? T(-1) : T(1);
    const T s11 = srow * scol;
    const bool own = own_c && y >= seg_lo && y < seg_hi && y < nf;
    const int zwo = zro + zc;
    ZGroup<TZ> zo;
    TZ zlo = TZ(0.0f);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int k = K0 + b, i = k % 3, j = k / 3;
      const T bi0 = (i == 0) ? T(0.25) : (i == 1 ? s2q : T(-0.25));
      const T bi1 = (i == 1) ? T(0) : T(0.5);
      const T bi2 = (i == 0) ? T(0.25) : (i == 1 ? -s2q : T(-0.25));
      T a = bi0 * hr[0][j] + bi2 * hr[2 * D][j];
      if (i != 1) a += bi1 * hr[D][j];
      const int pos = 3 * i + j - 1;              // place in the group ((0,0): low-pass)
      const T zv = (i == 0 && j == 0) ? T(ld_z(&zl[kq])) : T(ld_z(&zq[RING > 0 ? 0 : kq].e[pos]));
      const T zn = (i == 1 && j == 1) ? fma(zv, s11, a)
                 : (i == 1) ? fma(zv, srow, a) : (j == 1) ? fma(zv, scol, a) : zv + a;
      if (i == 0 && j == 0) zlo = to_z(zn, (TZ*)nullptr);
      else zo.e[pos] = to_z(zn, (TZ*)nullptr);
      const T xv = zn - fmin(fmax(zn, -mu), mu);     // S_mu
      pr[0][j] += bi0 * xv;
      if (i != 1) pr[D][j] += bi1 * xv;
      pr[2 * D][j] += bi2 * xv;
    }
    if (own) {
      uint4* dstz = reinterpret_cast<uint4*>(zout + (gbase + 8 * zwo));
#pragma unroll
      for (int v = 0; v < NV; ++v) dstz[v] = zo.v[v];
      if (TOP) zout[lbase + zwo] = zlo;
    }
    if (y + F3_PF < yc1) zload(y + F3_PF, kq);
    // row y - D has all its contributions: horizontal synthesis
    const int r = y - D;
    if (r >= yo0) {
      const T A = T(0.25) * pr[0][0] + s2q * pr[0][1] - T(0.25) * pr[0][2];
      const T B = T(0.5) * (pr[0][0] + pr[0][2]);
      const T C = T(0.25) * pr[0][0] - s2q * pr[0][1] - T(0.25) * pr[0][2];
      const T out = B + __shfl_down_sync(FULL, A, D) + __shfl_up_sync(FULL, C, D);
      if (LEV == 2 && L == 2) {
        // s_1 row r (lanes 2..29) -> (b0 x b0)^T s_1 row r - 1 (lanes 3..28)
        const T g = T(0.5) * out +
                    T(0.25) * (__shfl_up_sync(FULL, out, 1) + __shfl_down_sync(FULL, out, 1));
        gq[0] = gq[1]; gq[1] = gq[2]; gq[2] = g;
        if (r - 1 >= seg_lo && lane >= 3 && lane < 3 + F3_TX)
          f2s[(r - 1 - ty0) * F3_TX + (lane - 3)] = T(0.25) * (gq[0] + gq[2]) + T(0.5) * gq[1];
      } else {
        // level 1: f row r (lanes 1..26) = out + level-2 part
        if (lane >= 1 && lane < 1 + F3_TX) {
          T fv = out;
          if (L == 2) fv += f2s[(r - ty0) * F3_TX + (lane - 1)];
          if (r < nf && x < nf) fout[(size_t)r * nf + x] = fv;
        }
      }
    }
    // shift the rings
#pragma unroll
    for (int k = 0; k < 2 * D; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) { hr[k][j] = hr[k + 1][j]; pr[k][j] = pr[k + 1][j]; }
    pr[2 * D][0] = pr[2 * D][1] = pr[2 * D][2] = T(0);
  };
#pragma unroll 1
  for (int y = yc0; y < yc1; y += F3_PF) {
#pragma unroll
    for (int k = 0; k < F3_PF; ++k)
      if (y + k < yc1) step(y + k, k);
  }
  if constexpr (RING > 0) {
    if (bulk) {
      if (rg.bad) {
        // a wait gave up: wait (bounded) for the copies this level issued
        // from that row on, so none lands after the CTA has gone
        for (int i = first_bad; i < n_issued; ++i) {
          const int g = seq0 + i;
          mbar_wait(rg.bar + g % RING, (unsigned)(g / RING) & 1u);
        }
      }
      rg.seq = seq0 + nrows;
    } else {
      cp_wait<0>();
    }
    __syncwarp();
  }
}

template <typename T, typename TZ, int L, int F3_NWR, int F3_PF, int RING>
__global__ void __launch_bounds__(32 * F3_NWR)
k_frame3(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
         int u_slot, int f_slot, const void* zin_op, void* zout_op, double op_mu) {
  using Gm = F3<L, F3_NWR>;
  constexpr int F3_TY = Gm::TY;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  const State& st = states[item.x];
  if (st.stopped) return;
  const int nf = pd.nf;
  const int tilesX = (nf + F3_TX - 1) / F3_TX;
  const int ty0 = (item.y / tilesX) * F3_TY, tx0 = (item.y % tilesX) * F3_TX;
  const T mu = T(zin_op ? op_mu : pd.mu);
  const TZ* zin;
  TZ* zout;
  if (zin_op) {
    zin = static_cast<const TZ*>(zin_op);
    zout = static_cast<TZ*>(zout_op);
  } else {
    zin = static_cast<const TZ*>(pd.z[(st.iter - 1) & 1]);
    zout = static_cast<TZ*>(pd.z[st.iter & 1]);
  }
  T* su = reinterpret_cast<T*>(smraw);            // u on rows ty0 - C0.., cols tx0 - C0..
  T* sf2 = su + Gm::UW * Gm::UH;                  // level-2 part of f on the tile (L = 2)
  constexpr int C0 = Gm::C0;
  {
    int mode;
    const T* src;
    if (u_slot >= 0) { src = static_cast<const T*>(pd.buf[u_slot]); mode = 1; }
    else if (!pd.use_adj) { src = static_cast<const T*>(pd.buf[SL_T]); mode = 1; }
    else if (pd.bc == BC_RECT) { src = static_cast<const T*>(pd.buf[SL_V]); mode = 1; }
    else { src = static_cast<const T*>(pd.buf[SL_V]); mode = 0; }
    const bool interior = ty0 - C0 >= 0 && tx0 - C0 >= 0 && ty0 + F3_TY + C0 <= nf &&
                          tx0 + F3_TX + C0 <= nf;
    constexpr int NT = 32 * F3_NWR;
    constexpr int UN = Gm::UW * Gm::UH;
    // the BC fold of V has a single term wherever the tile keeps c pixels
    // from the image edges (or for zero BCs): u(a, b) = V(a + c, b + c)
    const int cc = pd.c;
    const bool single = mode == 0 && interior &&
                        (pd.bc == BC_ZERO || (ty0 - C0 >= cc && tx0 - C0 >= cc &&
                                              ty0 + F3_TY + C0 <= nf - cc && tx0 + F3_TX + C0 <= nf - cc));
    if (mode || single) {
      // plain copies of the (reflected) source: asynchronous, all of a
      // thread's copies in flight together, no registers held
      const int pitch = mode ? nf : pd.ne, off = mode ? 0 : cc;
      for (int idx = threadIdx.x; idx < UN; idx += NT) {
        const int ry = idx / Gm::UW, rx = idx - ry * Gm::UW;
        bool par;
        const int ay = interior ? ty0 - C0 + ry : f3_refl(ty0 - C0 + ry, nf, &par);
        const int ax = interior ? tx0 - C0 + rx : f3_refl(tx0 - C0 + rx, nf, &par);
        const T* g = src + ((size_t)(ay + off) * pitch + (ax + off));
        if (sizeof(T) == 8) cp_async_8(su + idx, g); else cp_async_4(su + idx, g);
      }
      cp_commit();
      cp_wait<0>();
    } else {
      // the BC fold of V sums up to four entries per element
      for (int idx = threadIdx.x; idx < UN; idx += NT) {
        const int ry = idx / Gm::UW, rx = idx - ry * Gm::UW;
        const int gy = ty0 - C0 + ry, gx = tx0 - C0 + rx;
        int o;
        const int ay = interior ? gy : refl_half(gy, nf, &o);
        const int ax = interior ? gx : refl_half(gx, nf, &o);
        su[idx] = fold_fetch<T>(pd, src, ay, ax);
      }
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int seg_lo = ty0 + w * F3_SEG, seg_hi = seg_lo + F3_SEG;
  if (seg_lo >= nf) return;        // no barrier follows
  T* f = static_cast<T*>(pd.buf[f_slot]);
  // this warp's ring of z rows and its mbarriers (RING > 0)
  F3Ring<TZ> rg;
  rg.seq = 0;
  rg.bad = false;
  rg.buf = nullptr;
  rg.bar = nullptr;
  if constexpr (RING > 0) {
    unsigned char* rb = smraw + frame3_ring_offset<T, TZ, L, F3_NWR, RING>();
    rg.buf = reinterpret_cast<TZ*>(rb + (size_t)w * RING * f3_slot_bytes<TZ>());
    rg.bar = reinterpret_cast<unsigned long long*>(rb + (size_t)F3_NWR * RING * f3_slot_bytes<TZ>()) +
             w * RING;
    if ((threadIdx.x & 31) == 0) {
      for (int k = 0; k < RING; ++k) mbar_init(rg.bar + k, 1);
      mbar_init_fence();
    }
    __syncwarp();
  }
  if (L == 2) {
    f3_level<T, TZ, 2, L, F3_PF, RING>(pd, su, Gm::UW, ty0 - C0, tx0 - C0, zin, zout, ty0, tx0,
                                       seg_lo, seg_hi, mu, sf2, f, rg);
    __syncwarp();
  }
  if (!rg.bad)
    f3_level<T, TZ, 1, L, F3_PF, RING>(pd, su, Gm::UW, ty0 - C0, tx0 - C0, zin, zout, ty0, tx0,
                                       seg_lo, seg_hi, mu, sf2, f, rg);
  if (rg.bad && (threadIdx.x & 31) == 0) {
    // a bounded wait gave up: the problem stops with a timeout status
    volatile State* vs = &states[item.x];
    vs->status = -4;
    vs->stopped = 1;
  }
}

int frame_tiles(int nf, int levels, int shape) {
  if (levels <= 2) {
    const int ty = F3_SEG * F3_SHAPES[shape].nwr;
    return ((nf + F3_TX - 1) / F3_TX) * ((nf + ty - 1) / ty);
  }
  return ((nf + FRAME_TILE - 1) / FRAME_TILE) * ((nf + FRAME_TILE - 1) / FRAME_TILE);
}

void frame_shape(int shape, int* tile_x, int* tile_y, int* prefetch) {
  *tile_x = F3_TX;
  *tile_y = F3_SEG * F3_SHAPES[shape].nwr;
  *prefetch = F3_SHAPES[shape].ring > 0 ? F3_SHAPES[shape].ring : F3_SHAPES[shape].pf;
}

// Planar (band-major) <-> grouped z layout (L <= 2), element size E bytes.
template <typename E>
__global__ void k_zlayout(E* __restrict__ dst, const E* __restrict__ src, int nbands, int plane,
                          int to_grouped) {
  const size_t tot = (size_t)nbands * plane;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / plane), q = (int)(i - (size_t)b * plane);
    const size_t g = (b < nbands - 1) ? (size_t)(b / 8) * 8 * plane + (size_t)8 * q + (b % 8) : i;
    if (to_grouped) dst[g] = src[i]; else dst[i] = src[g];
  }
}

bool z_grouped(int levels) { return levels <= 2; }

size_t z_grouped_index(int b, size_t q, int nbands, size_t plane) {
  return (b < nbands - 1) ? (size_t)(b / 8) * 8 * plane + 8 * q + (b % 8) : (size_t)b * plane + q;
}

void launch_z_layout(void* dst, const void* src, int levels, int nf, int elem_bytes,
                     int to_grouped, cudaStream_t s) {
  const int nbands = 8 * levels + 1, plane = nf * nf;
  const size_t tot = (size_t)nbands * plane;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (elem_bytes == 8)
    k_zlayout<unsigned long long><<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(dst),
        static_cast<const unsigned long long*>(src), nbands, plane, to_grouped);
  else if (elem_bytes == 4)
    k_zlayout<unsigned int><<<blocks, 256, 0, s>>>(static_cast<unsigned int*>(dst),
        static_cast<const unsigned int*>(src), nbands, plane, to_grouped);
  else
    k_zlayout<unsigned short><<<blocks, 256, 0, s>>>(static_cast<unsigned short*>(dst),
        static_cast<const unsigned short*>(src), nbands, plane, to_grouped);
}

// the kernel of one tile shape, its shared memory and its launch (FP64 has
// only shape 0); the cases follow F3_SHAPES
#define F3_SHAPE_CASES(X) \
  X(1, 1, 2, 0) X(2, 4, 2, 0) X(3, 2, 3, 0) X(4, 1, 3, 0) X(5, 2, 2, 6) X(6, 2, 2, 10) X(7, 1, 2, 12)

template <typename T, typename TZ, int L>
const void* frame3_kernel(int shape) {
  if constexpr (sizeof(T) == 8) {
    return (const void*)k_frame3<T, TZ, L, 2, 2, 0>;
  } else {
    switch (shape) {
#define X(S, NWR, PF, RING) case S: return (const void*)k_frame3<T, TZ, L, NWR, PF, RING>;
      F3_SHAPE_CASES(X)
#undef X
      default: return (const void*)k_frame3<T, TZ, L, 2, 2, 0>;
    }
  }
}
template <typename T, typename TZ, int L>
size_t frame3_smem(int shape) {
  if constexpr (sizeof(T) == 8) {
    return frame3_smem_bytes<T, TZ, L, 2, 0>();
  } else {
    switch (shape) {
#define X(S, NWR, PF, RING) case S: return frame3_smem_bytes<T, TZ, L, NWR, RING>();
      F3_SHAPE_CASES(X)
#undef X
      default: return frame3_smem_bytes<T, TZ, L, 2, 0>();
    }
  }
}
template <typename T, typename TZ, int L>
void launch_frame3_shape(int shape, const Prob* probs, State* states, const int2* items, int nitems,
                         int u_slot, int f_slot, const void* zin, void* zout, double op_mu,
                         cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    k_frame3<T, TZ, L, 2, 2, 0><<<nitems, 64, frame3_smem_bytes<T, TZ, L, 2, 0>(), s>>>(
        probs, states, items, u_slot, f_slot, zin, zout, op_mu);
  } else {
    switch (shape) {
#define X(S, NWR, PF, RING)                                                                     \
  case S:                                                                                       \
    k_frame3<T, TZ, L, NWR, PF, RING><<<nitems, 32 * NWR, frame3_smem_bytes<T, TZ, L, NWR, RING>(), s>>>( \
        probs, states, items, u_slot, f_slot, zin, zout, op_mu);                               \
    break;
      F3_SHAPE_CASES(X)
#undef X
      default:
        k_frame3<T, TZ, L, 2, 2, 0><<<nitems, 64, frame3_smem_bytes<T, TZ, L, 2, 0>(), s>>>(
            probs, states, items, u_slot, f_slot, zin, zout, op_mu);
    }
  }
}

template <typename T, typename TZ>
void launch_frame(const Prob* probs, State* states, const int2* items, int nitems, int u_slot,
                  int f_slot, const void* zin, void* zout, double op_mu, size_t smem, int levels,
                  int shape, cudaStream_t s) {
  if (nitems <= 0) return;
  if (levels == 1)
    launch_frame3_shape<T, TZ, 1>(shape, probs, states, items, nitems, u_slot, f_slot, zin, zout, op_mu, s);
  else if (levels == 2)
    launch_frame3_shape<T, TZ, 2>(shape, probs, states, items, nitems, u_slot, f_slot, zin, zout, op_mu, s);
  else
    k_frame<T, TZ><<<nitems, FRAME_THREADS, smem, s>>>(probs, states, items, u_slot, f_slot, zin,
                                                         zout, op_mu);
}
template <typename T, typename TZ>
cudaError_t frame_set_smem(size_t bytes) {
  for (int sh = 0; sh < FRAME_SHAPES; ++sh) {
    cudaError_t e = cudaFuncSetAttribute(frame3_kernel<T, TZ, 1>(sh),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)frame3_smem<T, TZ, 1>(sh));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(frame3_kernel<T, TZ, 2>(sh), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)frame3_smem<T, TZ, 2>(sh));
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_frame<T, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

bool is_frame_kernel(const void* func) {
  for (int sh = 0; sh < FRAME_SHAPES; ++sh) {
    const void* k[] = {frame3_kernel<float, float, 1>(sh), frame3_kernel<float, float, 2>(sh),
                       frame3_kernel<float, __nv_bfloat16, 1>(sh), frame3_kernel<float, __nv_bfloat16, 2>(sh),
                       frame3_kernel<double, double, 1>(sh), frame3_kernel<double, double, 2>(sh)};
    for (const void* f : k)
      if (f == func) return true;
  }
  return func == (const void*)k_frame<float, float> || func == (const void*)k_frame<float, __nv_bfloat16> ||
         func == (const void*)k_frame<double, double>;
}

#define INST(T, TZ)                                                                          \
  template size_t frame_smem_bytes<T, TZ>(int);                                              \
  template void launch_frame<T, TZ>(const Prob*, State*, const int2*, int, int, int,          \
                                    const void*, void*, double, size_t, int, int,             \
                                    cudaStream_t);                                            \
  template cudaError_t frame_set_smem<T, TZ>(size_t);
INST(float, float)
INST(float, __nv_bfloat16)
INST(double, double)
#undef INST

}  // namespace mlba
