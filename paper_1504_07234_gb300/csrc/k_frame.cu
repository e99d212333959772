// k_frame.cu — fused undecimated B-spline framelet step of Eq. MLBA2:
//
//     z_out = z_in + W u,   x = S_mu(z_out),   f = W^T x
//
// W is the L-level undecimated transform of Section 6.1 (masks b0, b1, b2,
// dilated by 2^(l-1) at level l, half-sample reflective boundary).  All
// values are computed on the reflectively extended domain around a tile: z
// outside the image is its mirror image with the sign of the band's symmetry
// (b1 is antisymmetric).  The extension of W u under the same mirroring
// equals W of the extended u, and S_mu is odd, so every value on a halo is
// exact and W^T reduces to plain (dilated) convolutions there.  z is read from
// one ping-pong buffer and written to the other (no in-place race between
// neighbouring tiles), once per owned coefficient.
//
// Two kernel families: for L <= 2 one fused row sweep per tile (k_frame3);
// for L >= 3 a low-pass chain and one row-sweep kernel per level, which works
// in the polyphase order of its dilation so that its halo is one position
// (k_lowpass, k_frame_lev).
//
// u comes from (per problem): the full correlation V folded by the BC
// transpose (A^T t for imposed boundary conditions), V itself (rectangular
// A), or t (Algorithm 4 forms, where C^T is already applied).
#include "mlba_internal.cuh"
#include "mlba_launch.h"

namespace mlba {

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
// rows past the register queue whose z lines are prefetched into L2: the
// queue holds PF rows in registers, the prefetch reaches further without
// holding any (measured on the 64-problem batch and on L = 4: 0.61 -> 0.51 ms
// per framelet launch; distances 1..10 tried)
constexpr int Z_L2_AHEAD = 2;   // k_frame3
constexpr int LV_L2_AHEAD = 1;  // k_frame_lev
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
  // owned rows [seg_lo, own_hi): one unsigned compare per row
  const unsigned own_rows = (unsigned)max(min(seg_hi, nf) - seg_lo, 0);
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
  // each queued row's mirrored offset and mirroring parity, mapped once when
  // the row is queued and used again when it is swept
  int zqo[F3_PF];
  bool zqp[F3_PF];
  // (idle lanes load a valid mirrored column too; their values are unused.
  // Offsets stay in 32 bits: nbands nf^2 < 2^31.)
  auto zload = [&](int y, int k) {
    bool par;
    const int q = f3_refl(y, nf, &par) * nf + zc;
    zqo[k] = q;
    zqp[k] = par;
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
    // z outside the image is its mirror image; antisymmetric (b1) bands
    // change sign under an odd number of mirrorings
    const T srow = zqp[kq] ? T(-1) : T(1);
    const T s11 = srow * scol;
    const bool own = own_c && (unsigned)(y - seg_lo) < own_rows;
    const int zwo = zqo[kq];
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
    if constexpr (RING == 0) {
      // the z lines of a row further ahead into L2 (no registers held): the
      // register queue then finds them there
      const int ya = y + F3_PF + Z_L2_AHEAD;
      if (ya < yc1) {
        // (ya >= 0; past the bottom edge the row is clamped rather than
        // mirrored: a prefetch of a neighbouring line only costs an L2 miss)
        const int qa = min(ya, nf - 1) * nf + zc;
        prefetch_l2(zin + (gbase + 8 * qa));
        if (TOP) prefetch_l2(zin + (lbase + qa));
      }
    }
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

// One framelet tile on the thread group `blk` of 32 F3_NWR threads with its
// shared memory at smraw.
template <typename T, typename TZ, int L, int F3_NWR, int F3_PF, int RING, typename BLK>
__device__ __forceinline__ void frame3_body(const int2 item, const Prob* __restrict__ probs,
                                            State* __restrict__ states, int u_slot, int f_slot,
                                            const void* zin_op, void* zout_op, double op_mu,
                                            unsigned char* smraw, BLK blk) {
  const int tid = blk.tid();
  using Gm = F3<L, F3_NWR>;
  constexpr int F3_TY = Gm::TY;
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
    zin = static_cast<const TZ*>(pd.z0 ? pd.z0 : pd.z[(st.iter - 1) & 1]);
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
    else if (pd.bc == BC_AR || pd.balanced) { src = static_cast<const T*>(pd.buf[SL_U]); mode = 1; }   // A' t; f + u
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
      for (int idx = tid; idx < UN; idx += NT) {
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
      for (int idx = tid; idx < UN; idx += NT) {
        const int ry = idx / Gm::UW, rx = idx - ry * Gm::UW;
        const int gy = ty0 - C0 + ry, gx = tx0 - C0 + rx;
        int o;
        const int ay = interior ? gy : refl_half(gy, nf, &o);
        const int ax = interior ? gx : refl_half(gx, nf, &o);
        su[idx] = fold_fetch<T>(pd, src, ay, ax);
      }
    }
  }
  blk.sync();
  const int w = tid >> 5;
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
    if ((tid & 31) == 0) {
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
  if (rg.bad && (tid & 31) == 0) {
    // a bounded wait gave up: the problem stops with a timeout status
    volatile State* vs = &states[item.x];
    vs->status = -4;
    vs->stopped = 1;
  }
}
template <typename T, typename TZ, int L, int F3_NWR, int F3_PF, int RING>
__global__ void __launch_bounds__(32 * F3_NWR)
k_frame3(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
         int u_slot, int f_slot, const void* zin_op, void* zout_op, double op_mu) {
  extern __shared__ __align__(16) unsigned char smraw[];
  frame3_body<T, TZ, L, F3_NWR, F3_PF, RING>(items[blockIdx.x], probs, states, u_slot, f_slot, zin_op,
                                             zout_op, op_mu, smraw, BlkFull{});
}


// ---------------------------------------------------------------------------
// L >= 3: the step level by level (the paper's experiments use L = 4).
//
//   c_0 = u,  c_l = (b0 x b0)_{2^(l-1)} c_{l-1}         (k_lowpass, kept in HBM)
//   level l = L, L-1, ..., 1 (k_frame_lev, dilation D = 2^(l-1)):
//     z_l <- z_l + W_l c_{l-1},  x = S_mu(z_l),
//     s_{l-1} = sum over the level's bands of B_ij^T x_ij  +  (b0 x b0)^T s_l
//   (the top level's nine bands include the final low-pass and it has no
//   s_L term), f = s_0.  s_1 .. s_{L-1} live in HBM too, so each kernel needs
//   a halo of its own dilation only (the fused single-pass form needs
//   2 (2^L - 1) = 30 pixels per side at L = 4), and in the polyphase order of
//   that dilation (Poly) the halo is one position: c_{l-1}, s_l and the
//   level's z are kept in the order of 2^(l-1), s_{l-1} in that of 2^(l-2).

// u as the level-1 kernel and the first low-pass read it: the op entry
// point's slot, t (Algorithm 4 forms), V (rectangular A), or U: the BC fold
// of V materialised before the sweep, or A' t for antireflective BCs
template <typename T>
__device__ __forceinline__ const T* frame_u(const Prob& pd, int u_slot) {
  if (u_slot >= 0) return static_cast<const T*>(pd.buf[u_slot]);
  if (!pd.use_adj) return static_cast<const T*>(pd.buf[SL_T]);
  if (pd.bc == BC_RECT) return static_cast<const T*>(pd.buf[SL_V]);
  return static_cast<const T*>(pd.buf[SL_U]);     // (also f + u of the balanced form)
}

// c_lev = (b0 x b0) with dilation d = 2^(lev-1) applied to c_{lev-1}, half-
// sample mirror at the border.  c_{lev-1} is read in the polyphase order of d
// (u, lev = 1: plain) and c_lev is written in that of 2d, the order of the
// kernels that read it.  The launch walks the input order: item.y = input
// row; for each column sub-lattice a of d the threads stride along it, its
// taps d apart being its neighbouring positions (contiguous reads), and its
// even and odd positions land in the output sub-lattices a and a + d (two
// contiguous runs of writes).
template <typename T>
__global__ void __launch_bounds__(LP_THREADS)
k_lowpass(const Prob* __restrict__ probs, const State* __restrict__ states,
          const int2* __restrict__ items, int lev, int u_slot) {
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  if (states[item.x].stopped) return;
  const int nf = pd.nf;
  const size_t plane = (size_t)nf * nf;
  const int d = 1 << (lev - 1);
  const Poly pin(nf, d), pout(nf, 2 * d);
  const T* in = (lev == 1) ? frame_u<T>(pd, u_slot)
                           : static_cast<const T*>(pd.lp) + (size_t)(lev - 2) * plane;
  const int iy = item.y;
  const int y = pin.inv(iy);
  bool par;
  const T* rm = in + (size_t)pin.pos(f3_refl(y - d, nf, &par)) * nf;
  const T* r0 = in + (size_t)iy * nf;
  const T* rp = in + (size_t)pin.pos(f3_refl(y + d, nf, &par)) * nf;
  T* out = static_cast<T*>(pd.lp) + (size_t)(lev - 1) * plane + (size_t)pout.pos(y) * nf;
  // the three input rows into L2 first (the sweep below then finds them there)
  prefetch_range(rm, (size_t)nf * sizeof(T), threadIdx.x, LP_THREADS);
  prefetch_range(r0, (size_t)nf * sizeof(T), threadIdx.x, LP_THREADS);
  prefetch_range(rp, (size_t)nf * sizeof(T), threadIdx.x, LP_THREADS);
  for (int a = 0; a < d; ++a) {
    const int ma = pin.count(a), sa = pin.start(a);
    // output run starts of the even and odd positions of sub-lattice a
    const int oe = a < nf ? pout.pos(a) : 0, oo = (a + d < nf) ? pout.pos(a + d) : 0;
#pragma unroll 4
    for (int m = threadIdx.x; m < ma; m += LP_THREADS) {
      const int ic = sa + m;
      int im = ic - 1, ip = ic + 1;             // neighbours inside the sub-lattice
      if (m == 0) im = pin.pos(f3_refl(a - d, nf, &par));
      if (m == ma - 1) ip = pin.pos(f3_refl(a + d * (m + 1), nf, &par));
      auto row = [&](const T* q) { return T(0.25) * (q[im] + q[ip]) + T(0.5) * q[ic]; };
      const T v = T(0.25) * (row(rm) + row(rp)) + T(0.5) * row(r0);
      out[(m & 1) ? oo + (m >> 1) : oe + (m >> 1)] = v;
    }
  }
}

// Level kernel geometry.  A level of dilation dp works in the polyphase
// order of dp (Poly): the taps dp apart join neighbouring positions m - 1, m,
// m + 1 of one sub-lattice, so the kernel runs the dilation-1 sweep on each
// of the dp^2 sub-lattices (a, b) (columns x = a + dp m, rows y = b + dp m).
// A CTA of LV_NWR warps owns OUTW positions of a column sub-lattice x 32
// LV_NWR positions of a row sub-lattice; lane k of a warp owns the
// coefficient column m = tx0 - 1 + k (every lane computes coefficients, lanes
// 1 .. 30 produce output).  The halo is one position whatever dp is.
struct LV {
  static constexpr int OUTW = 30;                 // output columns of a tile
  static constexpr int TY = 32 * LV_NWR;
  static constexpr int CW = 34, CH = TY + 4;      // c tile: positions tx0 - 2.., ty0 - 2..
  static constexpr int PR = 3;                    // synthesis ring rows
};
template <typename T>
__host__ __device__ constexpr size_t lev_smem_bytes() {
  return ((size_t)LV::CW * LV::CH + (size_t)LV_NWR * LV::PR * 3 * 32) * sizeof(T);
}
// tiles of one sub-lattice pair and of the whole level
__host__ __device__ inline void lev_tile_grid(int nf, int dp, int* tx, int* ty) {
  const int m = Poly(nf, dp).count_max();
  *tx = (m + LV::OUTW - 1) / LV::OUTW;
  *ty = (m + LV::TY - 1) / LV::TY;
}

// One level of the step.  The warp sweeps down its rows (one row
// sub-lattice): the horizontal analysis of the three rows m - 1, m, m + 1 of
// c_{l-1} (shared-memory tile, polyphase order of dp), the vertical masks,
// the update of z (register queue, PF rows ahead; z of the level in the same
// order), the threshold, and the vertical synthesis scattered into a ring of
// three rows (shared memory, one column per lane); row m - 1 then has all
// its contributions and is combined horizontally by warp shuffles at +-1 and,
// for l < L, with (b0 x b0)^T s_l: each lane loads s_l at its own column
// with the z rows (PF rows ahead) and keeps the horizontally filtered rows
// m - 2 .. m in registers (shuffles at +-1).  s_{l-1} is written in the
// polyphase order of dp / 2 (f, and s_1, plainly).  Coefficients outside the
// image are mirrored with the sign of the band's symmetry, as in k_frame3.
template <typename T, typename TZ, bool TOP>
__global__ void __launch_bounds__(32 * LV_NWR)
k_frame_lev(const Prob* __restrict__ probs, State* __restrict__ states,
            const int2* __restrict__ items, int lev, int u_slot, int f_slot, const void* zin_op,
            void* zout_op, double op_mu) {
  using G = LV;
  constexpr int PF = 2;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int K0 = TOP ? 0 : 1;            // band k = 3 j + i; (0,0) only at the top level
  constexpr int NB = 9 - K0;
  constexpr int NV = 8 * (int)sizeof(TZ) / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  const State& st = states[item.x];
  if (st.stopped) return;
  const int nf = pd.nf, L = pd.levels;
  const int plane = nf * nf;                 // nbands nf^2 < 2^31 is checked at set-up
  const int dp = 1 << (lev - 1);
  const Poly P(nf, dp), PO(nf, dp > 1 ? dp / 2 : 1);
  int tX, tY;
  lev_tile_grid(nf, dp, &tX, &tY);
  int t = item.y;
  const int tx = t % tX;
  t /= tX;
  const int ty = t % tY;
  t /= tY;
  const int sa = t % dp, sb = t / dp;        // column and row sub-lattices
  const int Ma = P.count(sa), Mb = P.count(sb);
  const int tx0 = tx * G::OUTW, ty0 = ty * G::TY;
  if (tx0 >= Ma || ty0 >= Mb) return;        // an empty tile (uniform over the CTA)
  const T mu = T(zin_op ? op_mu : pd.mu);
  const TZ* zin;
  TZ* zout;
  if (zin_op) {
    zin = static_cast<const TZ*>(zin_op);
    zout = static_cast<TZ*>(zout_op);
  } else {
    zin = static_cast<const TZ*>(pd.z0 ? pd.z0 : pd.z[(st.iter - 1) & 1]);
    zout = static_cast<TZ*>(pd.z[st.iter & 1]);
  }
  // position of the local coordinate m of a sub-lattice in the level's order
  // (mirrored into the image first)
  auto cpos = [&](int m, int off, bool* par) { return P.pos(f3_refl(off + dp * m, nf, par)); };
  T* sc = reinterpret_cast<T*>(smraw);       // c_{l-1} on rows ty0 - 2.., cols tx0 - 2..
  T* sring = sc + G::CW * G::CH;             // per-warp synthesis rings
  {
    const T* cin = (lev == 1) ? frame_u<T>(pd, u_slot)
                              : static_cast<const T*>(pd.lp) + (size_t)(lev - 2) * plane;
    // one warp per tile row (the row's position mapped once), lanes along the
    // row (columns lane and lane + 32, mapped once per lane)
    static_assert(G::CW <= 64, "two columns per lane");
    const int wq = threadIdx.x >> 5, ln = threadIdx.x & 31;
    bool par;
    const int ax0 = cpos(tx0 - 2 + ln, sa, &par);
    const bool two = ln + 32 < G::CW;
    const int ax1 = two ? cpos(tx0 - 2 + ln + 32, sa, &par) : 0;
    for (int ry = wq; ry < G::CH; ry += LV_NWR) {
      const T* row = cin + (size_t)cpos(ty0 - 2 + ry, sb, &par) * nf;
      T* d = sc + ry * G::CW + ln;
      if (sizeof(T) == 8) cp_async_8(d, row + ax0); else cp_async_4(d, row + ax0);
      if (two) {
        if (sizeof(T) == 8) cp_async_8(d + 32, row + ax1); else cp_async_4(d + 32, row + ax1);
      }
    }
    cp_commit();
    for (int idx = threadIdx.x; idx < LV_NWR * G::PR * 3 * 32; idx += 32 * LV_NWR) sring[idx] = T(0);
    cp_wait<0>();
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg_lo = ty0 + 32 * w, seg_hi = seg_lo + 32;
  if (seg_lo >= Mb) return;                  // no barrier follows
  const T s2q = T(0.35355339059327376220);   // sqrt(2) / 4
  const int mx = tx0 - 1 + lane;             // this lane's coefficient column (local)
  bool pcx;
  const int zc = cpos(mx, sa, &pcx);
  const T scol = pcx ? T(-1) : T(1);
  const bool own_c = lane >= 1 && lane < 31 && mx < Ma;
  const int yc0 = seg_lo - 1, yc1 = seg_hi + 1;
  T* ring = sring + w * (G::PR * 3 * 32) + lane;    // (row slot k, j) at ring[(3 k + j) 32]
  const T* ccol = sc + (lane + 1);                  // c tile column of mx
  const int crow0 = ty0 - 2;
  const int gbase = (lev - 1) * 8 * plane, lbase = 8 * L * plane;
  T* dst = (lev == 1) ? static_cast<T*>(pd.buf[f_slot])
                      : static_cast<T*>(pd.sy) + (size_t)(lev - 2) * plane;
  const int dcol = (own_c) ? PO.pos(sa + dp * mx) : 0;   // output column in dst's order
  const T* sin = TOP ? nullptr : static_cast<const T*>(pd.sy) + (size_t)(lev - 1) * plane;
  ZGroup<TZ> zq[PF];
  TZ zl[PF];
  T sq[PF];
  int zqo[PF];                               // queued rows' offsets and parities
  bool zqp[PF];
  auto zload = [&](int y, int k) {
    bool par;
    const int q = cpos(y, sb, &par) * nf + zc;
    zqo[k] = q;
    zqp[k] = par;
    const uint4* src = reinterpret_cast<const uint4*>(zin + (gbase + 8 * q));
#pragma unroll
    for (int v = 0; v < NV; ++v) zq[k].v[v] = src[v];
    if (TOP) zl[k] = zin[lbase + q];
    else sq[k] = sin[q];                     // s_l at (y, mx), mirrored like z
  };
  // (b0 x b0)^T s_l: horizontally filtered s_l rows m - 2, m - 1 (registers)
  T hs2 = T(0), hs1 = T(0);
#pragma unroll
  for (int k = 0; k < PF; ++k) zload(yc0 + k, k);
  // ring slots of rows m - 1, m, m + 1 (advanced by one per row)
  int k0 = 0, k1 = 1, k2 = 2;
  auto step = [&](int y, int kq) {
    // horizontal analysis of rows y - 1, y, y + 1: h[s][j]
    T h[3][3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const T* r = ccol + (y + (s - 1) - crow0) * G::CW;
      const T cm = r[-1], c0 = r[0], cp = r[1];
      const T sp = cm + cp;
      h[s][0] = T(0.25) * sp + T(0.5) * c0;
      h[s][1] = s2q * (cm - cp);
      h[s][2] = T(0.5) * c0 - T(0.25) * sp;
    }
    const T srow = zqp[kq] ? T(-1) : T(1);
    const T s11 = srow * scol;
    const bool own = own_c && y >= seg_lo && y < seg_hi && y < Mb;
    const int zwo = zqo[kq];
    ZGroup<TZ> zo;
    TZ zlo = TZ(0.0f);
    T p0[3] = {T(0), T(0), T(0)}, p1[3] = {T(0), T(0), T(0)}, p2[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int k = K0 + b, i = k % 3, j = k / 3;
      const T bi0 = (i == 0) ? T(0.25) : (i == 1 ? s2q : T(-0.25));
      const T bi1 = (i == 1) ? T(0) : T(0.5);
      const T bi2 = (i == 0) ? T(0.25) : (i == 1 ? -s2q : T(-0.25));
      T a = bi0 * h[0][j] + bi2 * h[2][j];
      if (i != 1) a += bi1 * h[1][j];
      const int pos = 3 * i + j - 1;
      const T zv = (i == 0 && j == 0) ? T(ld_z(&zl[kq])) : T(ld_z(&zq[kq].e[pos]));
      const T zn = (i == 1 && j == 1) ? fma(zv, s11, a)
                 : (i == 1) ? fma(zv, srow, a) : (j == 1) ? fma(zv, scol, a) : zv + a;
      if (i == 0 && j == 0) zlo = to_z(zn, (TZ*)nullptr);
      else zo.e[pos] = to_z(zn, (TZ*)nullptr);
      const T xv = zn - fmin(fmax(zn, -mu), mu);     // S_mu
      p0[j] += bi0 * xv;
      if (i != 1) p1[j] += bi1 * xv;
      p2[j] += bi2 * xv;
    }
    if (own) {
      uint4* dz = reinterpret_cast<uint4*>(zout + (gbase + 8 * zwo));
#pragma unroll
      for (int v = 0; v < NV; ++v) dz[v] = zo.v[v];
      if (TOP) zout[lbase + zwo] = zlo;
    }
    T hs0 = T(0);
    if (!TOP) {
      const T sv = sq[kq];
      hs0 = T(0.25) * (__shfl_up_sync(FULL, sv, 1) + __shfl_down_sync(FULL, sv, 1)) + T(0.5) * sv;
    }
    if (y + PF < yc1) zload(y + PF, kq);
    {
      const int ya = y + PF + LV_L2_AHEAD;     // z (and s_l) lines further ahead into L2
      if (ya < yc1) {
        bool par;
        const int qa = cpos(ya, sb, &par) * nf + zc;
        prefetch_l2(zin + (gbase + 8 * qa));
        if (TOP) prefetch_l2(zin + (lbase + qa));
        else prefetch_l2(sin + qa);
      }
    }
    // scatter into rows y - 1, y, y + 1; row y - 1 is then complete
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ring[(3 * k1 + j) * 32] += p1[j];
      ring[(3 * k2 + j) * 32] += p2[j];
    }
    T Pj[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Pj[j] = ring[(3 * k0 + j) * 32] + p0[j];
      ring[(3 * k0 + j) * 32] = T(0);         // the slot becomes row y + 2
    }
    const int r = y - 1;
    const T A = T(0.25) * Pj[0] + s2q * Pj[1] - T(0.25) * Pj[2];
    const T B = T(0.5) * (Pj[0] + Pj[2]);
    const T C = T(0.25) * Pj[0] - s2q * Pj[1] - T(0.25) * Pj[2];
    T out = B + __shfl_down_sync(FULL, A, 1) + __shfl_up_sync(FULL, C, 1);
    if (r >= seg_lo && own_c && r < Mb) {
      // (b0 x b0)^T s_l at (r, mx): rows r - 1 = y - 2, r, r + 1 = y
      if (!TOP) out += T(0.25) * (hs2 + hs0) + T(0.5) * hs1;
      dst[(size_t)PO.pos(sb + dp * r) * nf + dcol] = out;
    }
    hs2 = hs1;
    hs1 = hs0;
    k0 = (k0 + 1 == G::PR) ? 0 : k0 + 1;
    k1 = (k1 + 1 == G::PR) ? 0 : k1 + 1;
    k2 = (k2 + 1 == G::PR) ? 0 : k2 + 1;
  };
#pragma unroll 1
  for (int y = yc0; y < yc1; y += PF) {
#pragma unroll
    for (int k = 0; k < PF; ++k)
      if (y + k < yc1) step(y + k, k);
  }
}

#ifndef MLBA_BODIES_ONLY  // launchers: not in the persistent kernel's unit
int lev_tiles(int nf, int lev) {
  const int dp = 1 << (lev - 1);
  int tx, ty;
  lev_tile_grid(nf, dp, &tx, &ty);
  return dp * dp * tx * ty;
}
int lowpass_blocks(int nf) { return nf; }

template <typename T, typename TZ>
void launch_frame_levels(const Prob* probs, State* states, const int2* items, const int* sec,
                         int levels, int u_slot, int f_slot, const void* zin, void* zout,
                         double op_mu, cudaStream_t s) {
  // sec: (offset, count) of the fold, low-pass and level-L .. level-1 sections
  if (u_slot < 0 && sec[1] > 0) launch_vec<T>(VEC_FOLD, probs, states, items + sec[0], sec[1], 0, s);
  if (sec[3] > 0)
    for (int l = 1; l < levels; ++l)
      k_lowpass<T><<<sec[3], LP_THREADS, 0, s>>>(probs, states, items + sec[2], l, u_slot);
  for (int k = 0; k < levels; ++k) {
    const int lev = levels - k, off = sec[4 + 2 * k], cnt = sec[5 + 2 * k];
    if (cnt <= 0) continue;
    const int2* it = items + off;
    if (lev == levels)
      k_frame_lev<T, TZ, true><<<cnt, 32 * LV_NWR, lev_smem_bytes<T>(), s>>>(
          probs, states, it, lev, u_slot, f_slot, zin, zout, op_mu);
    else
      k_frame_lev<T, TZ, false><<<cnt, 32 * LV_NWR, lev_smem_bytes<T>(), s>>>(
          probs, states, it, lev, u_slot, f_slot, zin, zout, op_mu);
  }
}

int frame_tiles(int nf, int levels, int shape) {
  const int ty = F3_SEG * F3_SHAPES[shape].nwr;
  (void)levels;
  return ((nf + F3_TX - 1) / F3_TX) * ((nf + ty - 1) / ty);
}

void frame_shape(int shape, int* tile_x, int* tile_y, int* prefetch) {
  *tile_x = F3_TX;
  *tile_y = F3_SEG * F3_SHAPES[shape].nwr;
  *prefetch = F3_SHAPES[shape].ring > 0 ? F3_SHAPES[shape].ring : F3_SHAPES[shape].pf;
}

// Planar (band-major) <-> internal z layout (z_index), element size E bytes.
template <typename E>
__global__ void k_zlayout(E* __restrict__ dst, const E* __restrict__ src, int levels, int nf,
                          int to_internal) {
  const size_t plane = (size_t)nf * nf;
  const size_t tot = (size_t)(8 * levels + 1) * plane;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / plane);
    const int q = (int)(i - (size_t)b * plane);
    const int y = q / nf, x = q - y * nf;
    const size_t g = z_index(b, y, x, levels, nf);
    if (to_internal) dst[g] = src[i]; else dst[i] = src[g];
  }
}

bool z_grouped(int levels) { (void)levels; return true; }

void launch_z_layout(void* dst, const void* src, int levels, int nf, int elem_bytes,
                     int to_grouped, cudaStream_t s) {
  const int nbands = 8 * levels + 1;
  const size_t tot = (size_t)nbands * nf * nf;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (elem_bytes == 8)
    k_zlayout<unsigned long long><<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(dst),
        static_cast<const unsigned long long*>(src), levels, nf, to_grouped);
  else if (elem_bytes == 4)
    k_zlayout<unsigned int><<<blocks, 256, 0, s>>>(static_cast<unsigned int*>(dst),
        static_cast<const unsigned int*>(src), levels, nf, to_grouped);
  else
    k_zlayout<unsigned short><<<blocks, 256, 0, s>>>(static_cast<unsigned short*>(dst),
        static_cast<const unsigned short*>(src), levels, nf, to_grouped);
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
void launch_frame(const Prob* probs, State* states, const int2* items, int nitems, const int* sec,
                  int u_slot, int f_slot, const void* zin, void* zout, double op_mu, int levels,
                  int shape, cudaStream_t s) {
  if (nitems <= 0) return;
  if (levels == 1)
    launch_frame3_shape<T, TZ, 1>(shape, probs, states, items, nitems, u_slot, f_slot, zin, zout, op_mu, s);
  else if (levels == 2)
    launch_frame3_shape<T, TZ, 2>(shape, probs, states, items, nitems, u_slot, f_slot, zin, zout, op_mu, s);
  else
    launch_frame_levels<T, TZ>(probs, states, items, sec, levels, u_slot, f_slot, zin, zout, op_mu, s);
}

// the level kernels of one precision (below the top level, the top level)
// and the low-pass chain kernel
template <typename T, typename TZ>
const void* const* lev_kernels() {
  static const void* const k[] = {(const void*)k_frame_lev<T, TZ, false>,
                                  (const void*)k_frame_lev<T, TZ, true>, (const void*)k_lowpass<T>};
  return k;
}

template <typename T, typename TZ>
cudaError_t frame_set_smem() {
  for (int sh = 0; sh < FRAME_SHAPES; ++sh) {
    cudaError_t e = cudaFuncSetAttribute(frame3_kernel<T, TZ, 1>(sh),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)frame3_smem<T, TZ, 1>(sh));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(frame3_kernel<T, TZ, 2>(sh), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)frame3_smem<T, TZ, 2>(sh));
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < 2; ++k) {
    const cudaError_t e = cudaFuncSetAttribute(lev_kernels<T, TZ>()[k],
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)lev_smem_bytes<T>());
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool is_frame_kernel(const void* func) {
  for (int sh = 0; sh < FRAME_SHAPES; ++sh) {
    const void* k[] = {frame3_kernel<float, float, 1>(sh), frame3_kernel<float, float, 2>(sh),
                       frame3_kernel<float, __nv_bfloat16, 1>(sh), frame3_kernel<float, __nv_bfloat16, 2>(sh),
                       frame3_kernel<double, double, 1>(sh), frame3_kernel<double, double, 2>(sh)};
    for (const void* f : k)
      if (f == func) return true;
  }
  for (int k = 0; k < 3; ++k)
    if (func == lev_kernels<float, float>()[k] || func == lev_kernels<float, __nv_bfloat16>()[k] ||
        func == lev_kernels<double, double>()[k])
      return true;
  return false;
}

#define INST(T, TZ)                                                                          \
  template void launch_frame<T, TZ>(const Prob*, State*, const int2*, int, const int*, int,   \
                                    int, const void*, void*, double, int, int, cudaStream_t); \
  template cudaError_t frame_set_smem<T, TZ>();
INST(float, float)
INST(float, __nv_bfloat16)
INST(double, double)
#undef INST

#endif  // MLBA_BODIES_ONLY

}  // namespace mlba
