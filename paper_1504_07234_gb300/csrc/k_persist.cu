// k_persist.cu — host side of the persistent step kernel (k_persist.cuh) and
// its instantiation for FP32 z.
#include "k_persist.cuh"

namespace mlba {

size_t persist_smem(int dtype_bytes, int zs_bytes, int levels, size_t smem_stencil, size_t smem_fft,
                    int* stencil_slot, int* frame_slot) {
  const size_t st = (smem_stencil + 15) / 16 * 16;
  size_t fr;
  if (zs_bytes == 2) fr = levels == 1 ? frame3_smem_bytes<float, __nv_bfloat16, 1, 2, 0>() : frame3_smem_bytes<float, __nv_bfloat16, 2, 2, 0>();
  else fr = levels == 1 ? frame3_smem_bytes<float, float, 1, 2, 0>() : frame3_smem_bytes<float, float, 2, 2, 0>();
  fr = (fr + 15) / 16 * 16;
  (void)dtype_bytes;
  *stencil_slot = (int)st;
  *frame_slot = (int)fr;
  return std::max(std::max(2 * st, 4 * fr), smem_fft);
}

const void* persist_func_bf16(int levels);   // k_persist_bf16.cu

// the kernel of the z storage type and level count (FP32 arithmetic)
const void* persist_func(int zs_bytes, int levels) {
  return zs_bytes == 2 ? persist_func_bf16(levels) : persist_func_tz<float>(levels);
}

cudaError_t launch_persist(int zs_bytes, int levels, int grid, size_t smem, const Prob* probs,
                           State* states, int nprob, const PersistStage* stages, int nst,
                           int ksteps, void* ctl, unsigned long long spin_ns, int stencil_slot,
                           int frame_slot, cudaStream_t s) {
  PersistCtl* c = static_cast<PersistCtl*>(ctl);
  void* args[] = {(void*)&probs, (void*)&states, (void*)&nprob, (void*)&stages, (void*)&nst,
                  (void*)&ksteps, (void*)&c, (void*)&spin_ns, (void*)&stencil_slot,
                  (void*)&frame_slot};
  const cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(PersistCtl), s);
  if (e != cudaSuccess) return e;
  // a cooperative launch: all CTAs resident at once (the grid barrier needs it)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, persist_func(zs_bytes, levels), args);
}

size_t persist_ctl_bytes() { return sizeof(PersistCtl); }
int persist_threads() { return PT; }

}  // namespace mlba
