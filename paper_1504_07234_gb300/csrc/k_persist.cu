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

// The persistent step as a graph: a memset of the barrier words, then the
// cooperative kernel for `ksteps` steps.  persist_graph builds it (the kernel
// node returned in knode); persist_graph_set_k changes the step count of an
// instantiated copy.
namespace {
struct PersistArgs {
  const Prob* probs;
  State* states;
  int nprob;
  const PersistStage* stages;
  int nst, ksteps;
  PersistCtl* ctl;
  unsigned long long spin_ns;
  int stencil_slot, frame_slot;
  void* args[10];
  cudaKernelNodeParams kp;
  PersistArgs(int zs_bytes, int levels, int grid, size_t smem, const Prob* p, State* st, int np,
              const PersistStage* sg, int ns, int k, void* c, unsigned long long spin, int ss,
              int fs)
      : probs(p), states(st), nprob(np), stages(sg), nst(ns), ksteps(k),
        ctl(static_cast<PersistCtl*>(c)), spin_ns(spin), stencil_slot(ss), frame_slot(fs) {
    void* a[10] = {(void*)&probs, (void*)&states, (void*)&nprob, (void*)&stages, (void*)&nst,
                   (void*)&ksteps, (void*)&ctl, (void*)&spin_ns, (void*)&stencil_slot,
                   (void*)&frame_slot};
    for (int i = 0; i < 10; ++i) args[i] = a[i];
    kp = cudaKernelNodeParams{};
    kp.func = const_cast<void*>(persist_func(zs_bytes, levels));
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(PT);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
  }
};
}  // namespace

cudaError_t persist_graph(int zs_bytes, int levels, int grid, size_t smem, const Prob* probs,
                          State* states, int nprob, const PersistStage* stages, int nst, int ksteps,
                          void* ctl, unsigned long long spin_ns, int stencil_slot, int frame_slot,
                          cudaGraph_t* g, cudaGraphNode_t* knode) {
  cudaError_t e = cudaGraphCreate(g, 0);
  if (e != cudaSuccess) return e;
  cudaMemsetParams ms = {};
  ms.dst = ctl;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = sizeof(PersistCtl) / 4;
  ms.height = 1;
  ms.pitch = sizeof(PersistCtl);
  cudaGraphNode_t mnode;
  e = cudaGraphAddMemsetNode(&mnode, *g, nullptr, 0, &ms);
  if (e != cudaSuccess) return e;
  PersistArgs a(zs_bytes, levels, grid, smem, probs, states, nprob, stages, nst, ksteps, ctl,
                spin_ns, stencil_slot, frame_slot);
  e = cudaGraphAddKernelNode(knode, *g, &mnode, 1, &a.kp);
  if (e != cudaSuccess) return e;
  // all CTAs resident at once (the grid barrier needs it)
  cudaLaunchAttributeValue v = {};
  v.cooperative = 1;
  return cudaGraphKernelNodeSetAttribute(*knode, cudaLaunchAttributeCooperative, &v);
}

cudaError_t persist_graph_set_k(cudaGraphExec_t x, cudaGraphNode_t knode, int zs_bytes, int levels,
                                int grid, size_t smem, const Prob* probs, State* states, int nprob,
                                const PersistStage* stages, int nst, int ksteps, void* ctl,
                                unsigned long long spin_ns, int stencil_slot, int frame_slot) {
  PersistArgs a(zs_bytes, levels, grid, smem, probs, states, nprob, stages, nst, ksteps, ctl,
                spin_ns, stencil_slot, frame_slot);
  return cudaGraphExecKernelNodeSetParams(x, knode, &a.kp);
}

size_t persist_ctl_bytes() { return sizeof(PersistCtl); }
int persist_threads() { return PT; }

}  // namespace mlba
