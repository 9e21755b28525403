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

// sin(pi t / 2) and cos(pi t / 2) for |t| <= 2^21, the frequency encoding's only
// transcendental.  Reduction (exact): q = t rounded to the nearest integer (adding
// 1.5 * 2^23 leaves q mod 4 in the low bits of the sum), u = t - q in [-1/2, 1/2].
// Then sin(pi u / 2) = u S(u^2) and cos(pi u / 2) = C(u^2) with S and C of degree 3:
// near-minimax relative-error fits on |u| <= 1/2 made for this encoding
// (reweighted least squares on a dense grid, coefficients rounded to FP32; fit
// error 3.3e-9 and 3.9e-8, FP32 evaluation within 1.7 ulp of sin and 1.5 ulp of
// cos over the whole interval).  The quadrant q mod 4 swaps the pair and sets the
// signs: sin(pi t / 2) = sin(q pi / 2 + pi u / 2).
__device__ __forceinline__ void nrc_sincospi_half(float t, float& s, float& c) {
  const float m = t + 12582912.0f;
  const float q = m - 12582912.0f;
  const float u = t - q;
  const float v = u * u;
  const float ps = fmaf(fmaf(fmaf(-4.601703025e-3f, v, 7.968004793e-2f), v, -0.6459634900f), v, 1.570796371f) * u;
  const float pc = fmaf(fmaf(fmaf(-2.041752636e-2f, v, 0.2536032796f), v, -1.233697653f), v, 1.0f);
  const uint32_t i = __float_as_uint(m);
  const float a = (i & 1u) ? pc : ps, b = (i & 1u) ? ps : pc;
  s = __uint_as_float(__float_as_uint(a) ^ ((i << 30) & 0x80000000u));
  c = __uint_as_float(__float_as_uint(b) ^ (((i + 1u) << 30) & 0x80000000u));
}

// x limited to [-2^15, 2^15] (NaN stays NaN), so that every octave's 2^(k+1) x lies
// in nrc_sincospi_half's domain; inside the box x is in [0, 1].
__device__ __forceinline__ float nrc_clamp(float x) {
  float y;
  asm("max.NaN.f32 %0, %1, 0fC7000000;\n\tmin.NaN.f32 %0, %0, 0f47000000;" : "=f"(y) : "f"(x));
  return y;
}

// One octave up: (sin a, cos a) -> (sin 2a, cos 2a) = (2 s c, c^2 - s^2).  In the
// form c^2 - s^2 (not 1 - 2 s^2) the step's Jacobian is twice a rotation, so an
// error already in the pair grows by exactly a factor 2 per octave, and each step
// adds at most 2^-25 to s and 2^-24 to c of FP32 rounding.  From the pair of
// nrc_sincospi_half (each within 2^-23), after k steps the pair is within
// 2^k * 4 * 2^-24 (Euclidean) of the exact pair of the same FP32 argument.
__device__ __forceinline__ void nrc_double_angle(float& s, float& c) {
  const float s2 = (s + s) * c;
  c = fmaf(c, c, -(s * s));
  s = s2;
}

// The 64-d encoding of one raw record as 32 BF16 pairs (feature 2m in the low half
// of word m).  Features:
//  0..35  position normalised to the box, axis j / 12, sin (even j) / cos (odd j)
//         of 2^((j % 12) / 2) pi x: six octaves per axis;
//  36..47 direction mapped to [0, 1] (x = (w + 1) / 2), axis (j - 36) / 4, two
//         octaves (pi x, 2 pi x);
//  48..59 the normal, same layout from 48;
//  60     roughness; 61..63 the constant 1.
// Octave 0 of every coordinate comes from nrc_sincospi_half, the higher octaves
// from nrc_double_angle.
//
// Words 0..17: the position's octaves.
__device__ __forceinline__ void nrc_encode_position(const float* raw, const float* lo, const float* inv_ext,
                                                    uint32_t* w) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float s, c;
    nrc_sincospi_half(nrc_clamp((raw[a] - lo[a]) * inv_ext[a]) * 2.0f, s, c);
    w[6 * a] = pack_bf16(s, c);
#pragma unroll
    for (int k = 1; k < 6; ++k) {
      nrc_double_angle(s, c);
      w[6 * a + k] = pack_bf16(s, c);
    }
  }
}

// Words 18..31 (written to w[0..13]): direction and normal octaves, roughness, ones.
__device__ __forceinline__ void nrc_encode_direction(const float* raw, uint32_t* w) {
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    float s, c;
    nrc_sincospi_half(nrc_clamp(0.5f * (raw[3 + a] + 1.0f)) * 2.0f, s, c);
    w[2 * a] = pack_bf16(s, c);
    nrc_double_angle(s, c);
    w[2 * a + 1] = pack_bf16(s, c);
  }
  w[12] = pack_bf16(raw[9], 1.0f);
  w[13] = pack_bf16(1.0f, 1.0f);
}

// All 32 words of one record (zeros when !live).
__device__ __forceinline__ void nrc_encode_packed(const float* raw, const float* lo, const float* inv_ext, bool live,
                                                  uint32_t (&w)[32]) {
  nrc_encode_position(raw, lo, inv_ext, w);
  nrc_encode_direction(raw, w + 18);
  if (!live) {
#pragma unroll
    for (int i = 0; i < 32; ++i) w[i] = 0u;
  }
}

}  // namespace ptgb
