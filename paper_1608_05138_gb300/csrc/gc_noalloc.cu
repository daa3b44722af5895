// gc_noalloc.cu -- a triangle-count entry point that allocates no memory.
//
// Callers that own a fixed memory arena, or that run where a device
// allocation may not happen at all (inside another allocator's callback,
// under a hard budget that forbids growth), cannot use gc_graph_upload: it
// allocates the CSR copy, the preparation arrays and the per-CTA tables. This entry point is a variant
// of the triangle step (Alg. 1: a Psi bitmap of Gamma(x), probed with the
// neighbours of each neighbour) that works directly on the caller's device
// CSR and writes the caller's device output. Its only scratch -- one bitmap
// per CTA marking Gamma(x) -- lives in a file-scope __device__ array that
// every GPU loading the library holds until the process exits:
//   kNoAllocCtas bitmaps x kNoAllocMaxN bits = 256 x 1,048,576 bits = 32 MiB.
// Graphs with more than kNoAllocMaxN vertices are rejected. A column index
// outside [0, n) is skipped (it would otherwise touch another CTA's bitmap).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr int32_t kNoAllocMaxN = 1 << 20;              // vertices
constexpr int kNoAllocCtas = 256;                      // CTAs, one bitmap each
constexpr int kNoAllocWords = kNoAllocMaxN / 32;       // 32-bit words per bitmap
constexpr int kNoAllocBlock = 512;

static __device__ __align__(256) uint32_t g_noalloc_scratch[(size_t)kNoAllocCtas * kNoAllocWords];

// Device address of g_noalloc_scratch, looked up once per device ordinal and
// kept for the life of the process: this assumes the device's primary context
// (the one the CUDA runtime uses) and no cudaDeviceReset in between, after
// which the cached address would name memory of a context that is gone.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};

// tri[p] = |Gamma(x) ∩ Gamma(ci[p])| for every slot p of row x. Rows are dealt
// round-robin to CTAs; each CTA marks Gamma(x) in its bitmap, counts marked
// neighbours of every y in Gamma(x) (one warp per y), then unmarks Gamma(x).
__global__ void __launch_bounds__(kNoAllocBlock) k_triangles_noalloc(int32_t n, const int32_t* __restrict__ rp,
                                                                     const int32_t* __restrict__ ci,
                                                                     int32_t* __restrict__ tri,
                                                                     uint32_t* __restrict__ scratch) {
  uint32_t* bm = scratch + (size_t)blockIdx.x * kNoAllocWords;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warps = kNoAllocBlock / 32;
  // the array keeps the previous call's contents: start from zero
  const int32_t words = (n + 31) / 32;
  for (int32_t i = threadIdx.x; i < words; i += kNoAllocBlock) bm[i] = 0u;
  __syncthreads();
  for (int32_t x = blockIdx.x; x < n; x += gridDim.x) {
    const int32_t xb = rp[x], xe = rp[x + 1];
    for (int32_t p = xb + threadIdx.x; p < xe; p += kNoAllocBlock) {
      const int32_t w = ci[p];
      if ((uint32_t)w < (uint32_t)n) atomicOr(&bm[w >> 5], 1u << (w & 31));
    }
    __syncthreads();
    for (int32_t p = xb + warp; p < xe; p += warps) {
      const int32_t y = ci[p];
      int c = 0;
      if ((uint32_t)y >= (uint32_t)n) {  // not a vertex: no row to scan
        if (lane == 0) tri[p] = 0;
        continue;
      }
      for (int32_t q = rp[y] + lane; q < rp[y + 1]; q += 32) {
        const int32_t w = ci[q];
        if ((uint32_t)w < (uint32_t)n) c += (bm[w >> 5] >> (w & 31)) & 1u;
      }
      for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if (lane == 0) tri[p] = c;
    }
    __syncthreads();
    for (int32_t p = xb + threadIdx.x; p < xe; p += kNoAllocBlock) {
      const int32_t w = ci[p];
      if ((uint32_t)w < (uint32_t)n) bm[w >> 5] = 0u;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace gc

using namespace gc;

extern "C" gc_status gc_edge_triangles_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                               int32_t* tri_out, void* stream) {
  if (n < 0 || (n > 0 && (!row_ptr || !col_idx || !tri_out))) {
    set_error("gc_edge_triangles_noalloc: bad arguments");
    return GC_ERR_ARG;
  }
  if (n > kNoAllocMaxN) {
    set_error("gc_edge_triangles_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
              std::to_string(kNoAllocMaxN) + " vertices");
    return GC_ERR_OVERFLOW;
  }
  if (n == 0) return GC_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("gc_edge_triangles_noalloc: device index out of range");
    return GC_ERR_ARG;
  }
  uint32_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device (the current one): resolve the host-side
      // symbol to the device address of the array
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  k_triangles_noalloc<<<kNoAllocCtas, kNoAllocBlock, 0, (cudaStream_t)stream>>>(n, row_ptr, col_idx, tri_out,
                                                                                  scratch);
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : cuda_fail(e, "k_triangles_noalloc");
}
