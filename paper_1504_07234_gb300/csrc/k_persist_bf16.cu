// k_persist_bf16.cu — the persistent step kernel (k_persist.cuh) for bf16 z.
#include "k_persist.cuh"

namespace mlba {

const void* persist_func_bf16(int levels) { return persist_func_tz<__nv_bfloat16>(levels); }

}  // namespace mlba
