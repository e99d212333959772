// mlba_noalloc.cu — an entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory budget
// that is fixed before it starts (an allocator owned by a host framework
// that forbids side allocations), callers that must not trigger the implicit
// device synchronisation of cudaMalloc/cudaFree in a latency-critical loop,
// and plug-ins whose host process owns all device memory.  For them this
// file provides a variant of the residual stencil
//
//     r = g - A f,   norm2 = ||r||^2 (FP64 accumulation)
//
// whose only scratch (one FP64 partial per 32 x 32 tile plus the
// last-block counter of the deterministic reduction) lives in a file-scope
// __device__ array of fixed size.  The caller passes every input and output
// as device memory.  The array exists once per device for the lifetime of
// the process and is shared by every call, so calls that overlap on the GPU
// (different streams, or graph replays in flight together) race on it.
#include <cuda_runtime.h>
#include <mutex>

#include "../../include/mlba.h"
#include "mlba_internal.cuh"

namespace {

constexpr int NA_TILE = 32;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_TILES = (MLBA_NOALLOC_MAX_N / NA_TILE) * (MLBA_NOALLOC_MAX_N / NA_TILE);

// partials[0 .. NA_MAX_TILES) and, after them, the arrival counter
static __device__ __align__(256) double mlba_noalloc_scratch[NA_MAX_TILES + 32];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of a __device__ array is not a device
// address).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MLBA_E_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, mlba_noalloc_scratch) != cudaSuccess || !p) return MLBA_E_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MLBA_OK;
}

__global__ void __launch_bounds__(NA_THREADS)
k_residual_noalloc(const float* __restrict__ f, const float* __restrict__ g,
                   const float* __restrict__ psf, int p, int n, int bc, float* __restrict__ r,
                   double* __restrict__ norm2, double* __restrict__ scratch, int ntiles) {
  extern __shared__ __align__(16) float na_sm[];
  __shared__ double red[32];
  __shared__ int is_last;
  const int c = (p - 1) / 2;
  const int R = NA_TILE + p - 1;
  const int nf = (bc == mlba::BC_RECT) ? n + p - 1 : n;
  float* s_h = na_sm;            // p x p PSF
  float* s_in = na_sm + p * p;   // R x R region of f padded by the boundary condition
  const int tilesX = (n + NA_TILE - 1) / NA_TILE;
  const int ty0 = (blockIdx.x / tilesX) * NA_TILE, tx0 = (blockIdx.x % tilesX) * NA_TILE;
  for (int k = threadIdx.x; k < p * p; k += NA_THREADS) s_h[k] = psf[k];
  for (int idx = threadIdx.x; idx < R * R; idx += NA_THREADS) {
    const int ry = idx / R, rx = idx - ry * R;
    const int ey = ty0 - c + ry, ex = tx0 - c + rx;
    float v = 0.f;
    if (bc == mlba::BC_RECT) {
      const int my = ey + c, mx = ex + c;
      if (my >= 0 && my < nf && mx >= 0 && mx < nf) v = f[(size_t)my * nf + mx];
    } else {
      const int iy = mlba::bc_map(ey, n, bc), ix = mlba::bc_map(ex, n, bc);
      if (iy >= 0 && ix >= 0) v = f[(size_t)iy * n + ix];
    }
    s_in[idx] = v;
  }
  __syncthreads();
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  double lacc = 0.0;   // every square and sum in FP64
  for (int q = 0; q < 4; ++q) {
    const int oy = ly + 8 * q;
    const int gy = ty0 + oy, gx = tx0 + lx;
    float acc = 0.f;
    // (A f)(i,j) = sum_{a,b} H[a][b] f_ext(i - (a - c), j - (b - c))
    for (int a = 0; a < p; ++a) {
      const float* row = s_in + (oy + p - 1 - a) * R + lx + p - 1;
      for (int b = 0; b < p; ++b) acc += s_h[a * p + b] * row[-b];
    }
    if (gy < n && gx < n) {
      const size_t o = (size_t)gy * n + gx;
      const float rv = g[o] - acc;
      r[o] = rv;
      lacc += (double)rv * rv;
    }
  }
  const double bs = mlba::block_sum<NA_THREADS>(lacc, red);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + NA_MAX_TILES);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = bs;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == (unsigned)(ntiles - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < ntiles; i += NA_THREADS) s += __ldcg(&scratch[i]);
  s = mlba::block_sum<NA_THREADS>(s, red);
  if (threadIdx.x == 0) {
    *norm2 = s;
    *counter = 0u;
  }
}

}  // namespace

extern "C" int mlba_residual_noalloc(const float* f, const float* g, const float* psf, int p,
                                     int n, int bc, float* r, double* norm2, void* stream) {
  if (!f || !g || !psf || !r || !norm2 || p < 1 || (p % 2) == 0 || n < p || bc < 0 || bc > 3)
    return MLBA_E_INVAL;
  if (n > MLBA_NOALLOC_MAX_N || p > MLBA_NOALLOC_MAX_P) return MLBA_E_UNSUPPORTED;
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != MLBA_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tiles = ((n + NA_TILE - 1) / NA_TILE) * ((n + NA_TILE - 1) / NA_TILE);
  // the arrival counter must start at zero; a previous call that did not
  // finish normally could have left it set
  if (cudaMemsetAsync(scratch + NA_MAX_TILES, 0, sizeof(unsigned int), s) != cudaSuccess)
    return MLBA_E_CUDA;
  const int R = NA_TILE + p - 1;
  const size_t smem = (size_t)(p * p + R * R) * sizeof(float);
  k_residual_noalloc<<<tiles, NA_THREADS, smem, s>>>(f, g, psf, p, n, bc, r, norm2, scratch, tiles);
  return cudaGetLastError() == cudaSuccess ? MLBA_OK : MLBA_E_CUDA;
}
