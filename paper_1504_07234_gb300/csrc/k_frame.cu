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

template <typename T, typename TZ>
void launch_frame(const Prob* probs, State* states, const int2* items, int nitems, int u_slot,
                  int f_slot, const void* zin, void* zout, double op_mu, size_t smem,
                  cudaStream_t s) {
  if (nitems > 0)
    k_frame<T, TZ><<<nitems, FRAME_THREADS, smem, s>>>(probs, states, items, u_slot, f_slot, zin,
                                                         zout, op_mu);
}
template <typename T, typename TZ>
cudaError_t frame_set_smem(size_t bytes) {
  return cudaFuncSetAttribute(k_frame<T, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

#define INST(T, TZ)                                                                          \
  template size_t frame_smem_bytes<T, TZ>(int);                                              \
  template void launch_frame<T, TZ>(const Prob*, State*, const int2*, int, int, int,          \
                                    const void*, void*, double, size_t, cudaStream_t);       \
  template cudaError_t frame_set_smem<T, TZ>(size_t);
INST(float, float)
INST(float, __nv_bfloat16)
INST(double, double)
#undef INST

}  // namespace mlba
