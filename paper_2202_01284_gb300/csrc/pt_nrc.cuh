// Radiance-cache MLP building blocks shared by the cache kernels and the
// megakernel's cache modes: feature layout, BF16 warp-level MMA fragments
// (mma.sync m16n8k16, FP32 accumulate) and the 64-d input encoding.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ptgb {

constexpr int NRC_W = 64;        // layer width
constexpr int NRC_HIDDEN = 5;    // 64x64 layers (the first consumes the encoding)
constexpr int NRC_OUT = 3;
constexpr int NRC_PARAMS = NRC_HIDDEN * NRC_W * NRC_W + NRC_OUT * NRC_W;  // 20,672
constexpr int NRC_RAW = 10;      // raw record: position[3], direction[3], normal[3], roughness
constexpr int NRC_LD = 72;       // padded shared-memory row (bf16 elements): conflict-free fragment loads

struct NrcBox {
  float lo[3], inv_ext[3];
};

// Inference on the tcgen05 tensor cores (pt_nrc_tc.cu); `status` receives
// PT_ERR_TIMEOUT if a bounded wait on the tensor core gave up.
int cache_infer_tc(const float* raw, float* rgb, long long n, const NrcBox& box, const __nv_bfloat16* Wb, int* status,
                   unsigned wait_limit, cudaStream_t st);
// Training forward + backward deltas on tcgen05 (pt_nrc_tc.cu): writes X[6][n][64],
// dZ[6][n][64] and adds the batch's loss, as nrc_train_fb_kernel.
int cache_train_fb_tc(const float* raw, const float* target, long long n, const NrcBox& box, const __nv_bfloat16* Wb,
                      __nv_bfloat16* X, __nv_bfloat16* dZ, float* loss, int* status, unsigned wait_limit,
                      cudaStream_t st);
// Weight gradients on tcgen05 (pt_nrc_tc.cu): dW_l += dZ_l^T X_l, split-K over
// blocks of `chunk` records, as nrc_wgrad_kernel.
int cache_wgrad_tc(const __nv_bfloat16* X, const __nv_bfloat16* dZ, long long n, long long chunk, float* dW,
                   int* status, unsigned wait_limit, cudaStream_t st);

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// D = A(16x16 bf16, row) * B(16x8 bf16, col) + C (fp32)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* smem_row) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const void* smem_row) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// One encoded feature j (0..63) of a raw record; p is normalised to the box.
// j <  36: position, axis j/12, frequency 2^((j%12)/2) pi, sin (even j) / cos (odd j)
// j <  48: direction mapped to [0,1], axis (j-36)/4, frequency 2^(((j-36)%4)/2) pi
// j <  60: normal, same layout from 48
// j == 60: roughness; j > 60: constant 1
__device__ __forceinline__ float nrc_feature(int j, const float* raw, const float* lo, const float* inv_ext) {
  float x;
  int k;
  if (j < 36) {
    const int a = j / 12;
    k = (j % 12) >> 1;
    x = (raw[a] - lo[a]) * inv_ext[a];
  } else if (j < 60) {
    const int v = j < 48 ? 0 : 1;
    const int jj = j - (v ? 48 : 36);
    const int a = jj >> 2;
    k = (jj & 3) >> 1;
    x = 0.5f * (raw[3 + 3 * v + a] + 1.0f);
  } else {
    return j == 60 ? raw[9] : 1.0f;
  }
  float s, c;
  sincospif(ldexpf(x, k), &s, &c);
  return (j & 1) ? c : s;
}

}  // namespace ptgb
