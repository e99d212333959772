// k_persist.cuh — one persistent launch for k steps of a batch.
//
// The step's stages (residual stencil, transform passes, alpha_n passes,
// adjoint stencil, balanced input, fused framelet sweep) are walked by one
// cooperative grid: every CTA takes the items of a stage in turn (two stencil
// tiles or four framelet tiles side by side on sub-blocks of the CTA, one
// transform block on the whole CTA), then all CTAs meet at a grid barrier
// before the next stage.  The items, the per-problem stop flags and the
// arithmetic are those of the graph schedule, so the iterates are the same.
// Every barrier wait is bounded (a global-timer limit); when one gives up, the
// grid records MLBA_E_TIMEOUT in every problem's state and returns.
// The stage bodies come from the stencil, transform and framelet sources,
// included here without their kernels' launchers (MLBA_BODIES_ONLY), so this
// unit compiles only the persistent kernel.  k_persist.cu instantiates it for
// FP32 z, k_persist_bf16.cu for bf16 z (two units compiled in parallel).
#pragma once
#define MLBA_BODIES_ONLY
#include "k_stencil.cu"
#include "k_fft.cu"
#include "k_frame.cu"

namespace mlba {

// barrier and error words of a batch (device memory, zeroed before a launch)
struct PersistCtl {
  unsigned count, gen;
  int err;
  int pad;
};

constexpr int PT = 256;                // threads of a persistent CTA

__device__ __forceinline__ unsigned long long p_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned p_ld_acquire(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned p_ld_relaxed(const unsigned* a) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// Grid-wide barrier with a bounded wait (spin_ns; 0: a CTA that is not the
// last to arrive gives up at once).  Thread 0 of each CTA arrives with an
// acquire-release add on the counter (releasing what the CTA wrote: the CTA
// barrier before it orders the other threads' writes); the last to arrive
// resets the counter and releases the generation word, the others poll it
// with acquire loads.  False when this or another CTA gave up.
static __device__ bool p_grid_sync(PersistCtl* ctl, unsigned long long spin_ns, int* ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = p_ld_relaxed(&ctl->gen);
    unsigned arrived;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(arrived) : "l"(&ctl->count) : "memory");
    if (arrived == gridDim.x - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&ctl->count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->gen) : "memory");
    } else if (spin_ns == 0) {
      ok = 0;
    } else {
      const unsigned long long t0 = p_now();
      unsigned it = 0;
      while (p_ld_acquire(&ctl->gen) == g) {
        if (p_ld_relaxed(reinterpret_cast<const unsigned*>(&ctl->err))) { ok = 0; break; }
        if ((++it & 63u) == 0 && p_now() - t0 > spin_ns) { ok = 0; break; }
        __nanosleep(20);
      }
    }
    if (!ok) atomicExch(&ctl->err, 1);
    if (p_ld_relaxed(reinterpret_cast<const unsigned*>(&ctl->err))) ok = 0;
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

template <typename T, typename TZ, int L>
__global__ void __launch_bounds__(PT, 2)
k_persist(const Prob* __restrict__ probs, State* __restrict__ states, int nprob,
          const PersistStage* __restrict__ stages, int nst, int ksteps, PersistCtl* ctl,
          unsigned long long spin_ns, int stencil_slot, int frame_slot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[4][32];
  __shared__ int flag[4];
  __shared__ int ok_sh;
  const int sub2 = threadIdx.x >> 7, sub4 = threadIdx.x >> 6;
  for (int step = 0; step < ksteps; ++step) {
    for (int si = 0; si < nst; ++si) {
      const PersistStage sg = stages[si];
      const int2* it = sg.items;
      const int cnt = sg.count;
      switch (sg.kind) {
        case PS_RESID:
        case PS_CORR:
        case PS_REBLUR:
          // two stencil tiles per pass, one per 128-thread half
          for (int u = blockIdx.x; 2 * u < cnt; u += gridDim.x) {
            const int i = 2 * u + sub2;
            if (i >= cnt) continue;
            unsigned char* sm = smraw + (size_t)sub2 * stencil_slot;
            const BlkSub<STENCIL_THREADS> b{1 + sub2};
            if (sg.kind == PS_RESID)
              stencil_body<T, ST_FWD_RESID>(it[i], probs, states, SL_F, SL_R, SL_G, 0, sm, red[sub2], &flag[sub2], b);
            else if (sg.kind == PS_CORR)
              stencil_body<T, ST_CORR>(it[i], probs, states, -1, SL_V, SL_V, 0, sm, red[sub2], &flag[sub2], b);
            else
              stencil_body<T, ST_REBLUR>(it[i], probs, states, -1, -1, SL_U, 0, sm, red[sub2], &flag[sub2], b);
            b.sync();   // the next item's tile loads overwrite this one's shared memory
          }
          break;
        case PS_FRAME:
          // four framelet tiles per pass, one per 64-thread quarter
          for (int u = blockIdx.x; 4 * u < cnt; u += gridDim.x) {
            const int i = 4 * u + sub4;
            if (i >= cnt) continue;
            const BlkSub<64> b{1 + sub4};
            frame3_body<T, TZ, L, 2, 2, 0>(it[i], probs, states, -1, SL_F, nullptr, nullptr, 0.0,
                                           smraw + (size_t)sub4 * frame_slot, b);
            b.sync();
          }
          break;
        case PS_ROWS_FWD:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { rows_fwd_body<T>(it[u], probs, states, SL_R, 0); __syncthreads(); }
          break;
        case PS_COLS_FUSED:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { cols_body<T, COL_FUSED>(it[u], probs, states, 0, 0.0, 0); __syncthreads(); }
          break;
        case PS_COLS_FWD:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { cols_body<T, COL_FWD>(it[u], probs, states, 0, 0.0, 0); __syncthreads(); }
          break;
        case PS_SPEC:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { spec_body<T>(it[u], probs, states); __syncthreads(); }
          break;
        case PS_COLS_NSINV:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { cols_body<T, COL_NS_INV>(it[u], probs, states, 0, 0.0, 0); __syncthreads(); }
          break;
        case PS_ROWS_INV:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { rows_inv_body<T>(it[u], probs, states, SL_T, 0); __syncthreads(); }
          break;
        case PS_BALANCE:
          for (int u = blockIdx.x; u < cnt; u += gridDim.x) { balance_body<T>(it[u], probs, states); __syncthreads(); }
          break;
        default:
          break;
      }
      if (sg.sync && !p_grid_sync(ctl, spin_ns, &ok_sh)) {
        // a barrier wait gave up: every problem stops with MLBA_E_TIMEOUT
        if (threadIdx.x == 0)
          for (int i = 0; i < nprob; ++i) {
            volatile State* vs = &states[i];
            vs->status = -4;
            vs->stopped = 1;
          }
        return;
      }
    }
  }
}

template <typename TZ>
const void* persist_func_tz(int levels) {
  return levels == 1 ? (const void*)k_persist<float, TZ, 1> : (const void*)k_persist<float, TZ, 2>;
}

}  // namespace mlba
