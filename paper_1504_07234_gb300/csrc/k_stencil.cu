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
#include "mlba_internal.cuh"
#include "mlba_launch.h"

namespace mlba {

// stop rule and iteration bookkeeping after ||r^n||^2 is known
// (Eq. discrpr; Algorithm 4-NS and Eq. Alg4_rev_12)
__device__ void finalize_residual(const Prob& pd, State& st, double sumsq) {
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

template <typename T, int MODE>
__global__ void __launch_bounds__(STENCIL_THREADS)
k_stencil(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
          int src_slot, int dst_slot, int aux_slot, int pcg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (skip(st, pcg)) return;

  constexpr bool CORR = (MODE == ST_CORR);
  const int n = pd.n, p = pd.p, c = pd.c;
  const int outN = CORR ? pd.ne : n;
  const int tilesX = (outN + 31) >> 5;
  const int ty0 = (item.y / tilesX) * 32, tx0 = (item.y % tilesX) * 32;
  const int R = 32 + p - 1;
  const int ntaps = pd.sep ? 0 : pd.ntaps;

  T* s_w = reinterpret_cast<T*>(smraw);          // ntaps weights (or 2p separable)
  const int nw = pd.sep ? 2 * p : ntaps;
  T* s_in = s_w + ((nw + 1) & ~1);               // R x R input region
  T* s_tmp = s_in + R * R;                        // R x 32 (separable)
  int* s_off = reinterpret_cast<int*>(s_tmp + (pd.sep ? R * 32 : 0));

  // src_slot < 0: the per-problem default operand (t, or r for P = I, in the
  // correlation; A^T p for the PCG product: V for rectangular A, U otherwise)
  if (src_slot < 0)
    src_slot = CORR ? (pd.precond == P_NONE ? SL_R : SL_T) : (pd.bc == BC_RECT ? SL_V : SL_U);
  const T* src = static_cast<const T*>(pd.buf[src_slot]);
  // taps
  if (pd.sep) {
    const T* hy = static_cast<const T*>(pd.hy);
    const T* hx = static_cast<const T*>(pd.hx);
    for (int k = threadIdx.x; k < p; k += blockDim.x) { s_w[k] = hy[k]; s_w[p + k] = hx[k]; }
  } else {
    const T* tw = static_cast<const T*>(pd.tap_w);
    for (int k = threadIdx.x; k < ntaps; k += blockDim.x) {
      s_w[k] = tw[k];
      const int dy = pd.tap_dy[k], dx = pd.tap_dx[k];
      s_off[k] = CORR ? (c + dy) * R + (c + dx) : (c - dy) * R + (c - dx);
    }
  }
  // input region
  const int oy0 = CORR ? ty0 - 2 * c : ty0 - c;
  const int ox0 = CORR ? tx0 - 2 * c : tx0 - c;
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int ry = idx / R, rx = idx - ry * R;
    const int ey = oy0 + ry, ex = ox0 + rx;
    T v = T(0);
    if (CORR) {
      if (ey >= 0 && ey < n && ex >= 0 && ex < n) v = src[(size_t)ey * n + ex];
    } else if (pd.bc == BC_RECT) {
      const int my = ey + c, mx = ex + c;
      if (my >= 0 && my < pd.nf && mx >= 0 && mx < pd.nf) v = src[(size_t)my * pd.nf + mx];
    } else {
      const int iy = bc_map(ey, n, pd.bc), ix = bc_map(ex, n, pd.bc);
      if (iy >= 0 && ix >= 0) v = src[(size_t)iy * n + ix];
    }
    s_in[idx] = v;
  }
  __syncthreads();
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;   // 32 x 8 threads
  if (pd.sep) {
    // horizontal pass over all R rows, then vertical
    for (int ry = ly; ry < R; ry += 8) {
      T acc = T(0);
      for (int k = 0; k < p; ++k) {
        const int dx = k - c;
        acc += s_w[p + k] * s_in[ry * R + lx + (CORR ? c + dx : c - dx)];
      }
      s_tmp[ry * 32 + lx] = acc;
    }
    __syncthreads();
  }
  double local = 0.0;
  T* dst = static_cast<T*>(pd.buf[dst_slot]);
  const T* aux = static_cast<const T*>(pd.buf[aux_slot]);
  T lacc = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int oy = ly + 8 * q;
    T acc = T(0);
    if (pd.sep) {
      for (int k = 0; k < p; ++k) {
        const int dy = k - c;
        acc += s_w[k] * s_tmp[(oy + (CORR ? c + dy : c - dy)) * 32 + lx];
      }
    } else {
      const T* base = s_in + oy * R + lx;
      for (int k = 0; k < ntaps; ++k) acc += s_w[k] * base[s_off[k]];
    }
    const int gy = ty0 + oy, gx = tx0 + lx;
    if (gy < outN && gx < outN) {
      const size_t o = (size_t)gy * outN + gx;
      if (MODE == ST_FWD_RESID) {
        const T r = aux[o] - acc;
        dst[o] = r;
        lacc += r * r;
      } else if (MODE == ST_FWD_PCGQ) {
        const T pv = aux[o];
        const T qv = acc + T(pd.alpha) * pv;
        dst[o] = qv;
        lacc += pv * qv;
      } else {
        dst[o] = acc;
      }
    }
  }
  if (MODE == ST_FWD_RESID || MODE == ST_FWD_PCGQ) {
    local = (double)lacc;
    const double bs = block_sum<STENCIL_THREADS>(local, red);
    double tot[1];
    const double vals[1] = {bs};
    if (last_block_reduce<STENCIL_THREADS, 1>(pd, st, item.y, pd.nblk_blur, vals, tot, red)) {
      if (threadIdx.x == 0) {
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
template <typename T>
void launch_stencil(int mode, const Prob* probs, State* states, const int2* items, int nitems,
                    int src, int dst, int aux, int pcg, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return;
  dim3 g(nitems), b(STENCIL_THREADS);
  switch (mode) {
    case ST_FWD_RESID: k_stencil<T, ST_FWD_RESID><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    case ST_FWD_STORE: k_stencil<T, ST_FWD_STORE><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
    case ST_FWD_PCGQ: k_stencil<T, ST_FWD_PCGQ><<<g, b, smem, s>>>(probs, states, items, src, dst, aux, pcg); break;
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
template void launch_vec<float>(int, const Prob*, State*, const int2*, int, int, cudaStream_t);
template void launch_vec<double>(int, const Prob*, State*, const int2*, int, int, cudaStream_t);

}  // namespace mlba
