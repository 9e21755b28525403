// Measurement probes for the roofline of the path tracer (sm_103a).
//
// The traversal fetches 80-byte BVH nodes and 48-byte triangles through L2 (the
// scene of the throughput workload is L2-resident), and the adjoint scatters its
// gradient terms with float and float4 atomics into L2 (Sec. 4.1: the reverse pass
// is dominated by atomic scatter-adds).  Neither roof is in the driver's peak
// table, so the library measures them itself with these two kernels:
//   * probe_read_kernel   -- L2-resident float4 reads (ld.global.cg: cached in L2,
//                            not L1), four independent loads in flight per thread;
//   * probe_atomic_kernel -- fire-and-forget adds of 1.0 (RED) to n_addr addresses,
//                            float or float4, address i*2654435761 mod n_addr
//                            (spread over a large buffer, or colliding on a few).

#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"

namespace ptgb {
namespace {

__global__ void __launch_bounds__(256) probe_read_kernel(const float4* __restrict__ buf, long long n, int passes,
                                                         float* __restrict__ sink) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.0f;
  for (int p = 0; p < passes; ++p) {
    long long i = t;
    for (; i + 3 * stride < n; i += 4 * stride) {
      const float4 a = __ldcg(&buf[i]);
      const float4 b = __ldcg(&buf[i + stride]);
      const float4 c = __ldcg(&buf[i + 2 * stride]);
      const float4 d = __ldcg(&buf[i + 3 * stride]);
      acc += (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w) + (c.x + c.y + c.z + c.w) + (d.x + d.y + d.z + d.w);
    }
    for (; i < n; i += stride) {
      const float4 a = __ldcg(&buf[i]);
      acc += a.x + a.y + a.z + a.w;
    }
  }
  // one add per warp keeps the loads alive; the sum itself is the read check
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(sink, acc);
}

template <int WIDTH>
__global__ void __launch_bounds__(256) probe_atomic_kernel(float* __restrict__ dst, long long n_addr, long long n_upd) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_upd; i += stride) {
    const long long a = (long long)(((unsigned long long)i * 2654435761ull) % (unsigned long long)n_addr);
    if constexpr (WIDTH == 4) atomicAdd(reinterpret_cast<float4*>(dst) + a, make_float4(1.f, 1.f, 1.f, 1.f));
    else atomicAdd(dst + a, 1.0f);
  }
}

int probe_grid(int per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * per_sm;
}

}  // namespace
}  // namespace ptgb

using namespace ptgb;

extern "C" int pt_probe_read(const void* buf, long long bytes, int passes, float* sink, void* stream) {
  if (!buf || !sink || bytes <= 0 || bytes % 16 || passes < 1 || ((uintptr_t)buf & 15u)) return PT_ERR_ARG;
  probe_read_kernel<<<probe_grid(8), 256, 0, (cudaStream_t)stream>>>(static_cast<const float4*>(buf), bytes / 16,
                                                                       passes, sink);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_probe_atomic(float* dst, long long n_addr, long long n_updates, int width, void* stream) {
  if (!dst || n_addr < 1 || n_updates < 0 || (width != 1 && width != 4)) return PT_ERR_ARG;
  if (width == 4 && ((uintptr_t)dst & 15u)) return PT_ERR_ARG;
  if (n_updates == 0) return PT_OK;
  const cudaStream_t cs = (cudaStream_t)stream;
  if (width == 4) probe_atomic_kernel<4><<<probe_grid(8), 256, 0, cs>>>(dst, n_addr, n_updates);
  else probe_atomic_kernel<1><<<probe_grid(8), 256, 0, cs>>>(dst, n_addr, n_updates);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
