// Learned radiance cache: fused BF16 tensor-core MLP inference, training
// (forward + backward deltas, weight gradients as a split-K reduction), Adam,
// and the C-ABI object that owns weights, optimiser state and buffers.
//
// Not part of the paper (it names caches only as a direction, Sec. 3.2); the
// network and loss follow Mueller et al. 2021 (Real-time Neural Radiance
// Caching): 64-d frequency encoding, 5 x 64 ReLU layers, 3 outputs, relative
// L2 loss, Adam.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pt_internal.h"
#include "pt_nrc.cuh"

namespace ptgb {

// ---------------------------------------------------------------- shared-memory weight images
struct NrcSmem {
  // hidden weights [l][o][i] and the head [o(8)][i], rows padded to NRC_LD
  static constexpr int W_ELEMS = NRC_HIDDEN * NRC_W * NRC_LD + 8 * NRC_LD;
};

// Copy the BF16 weights (global [5][64][64] + head [8][64]) into padded shared rows.
// With `transposed`, also write W^T per layer ([i][o]) and the head's transpose
// ([i][16], outputs 3..15 zero) after the direct image.
__device__ __forceinline__ void load_weights_smem(const __nv_bfloat16* __restrict__ Wg, __nv_bfloat16* s,
                                                  bool transposed) {
  const unsigned short* g = reinterpret_cast<const unsigned short*>(Wg);
  unsigned short* d = reinterpret_cast<unsigned short*>(s);
  for (int idx = threadIdx.x; idx < NRC_HIDDEN * NRC_W * NRC_W + 8 * NRC_W; idx += blockDim.x) {
    const int row = idx / NRC_W, col = idx % NRC_W;  // row = l*64 + o (head rows follow)
    d[row * NRC_LD + col] = g[idx];
  }
  if (transposed) {
    unsigned short* t = d + NrcSmem::W_ELEMS;
    for (int idx = threadIdx.x; idx < NRC_HIDDEN * NRC_W * NRC_W; idx += blockDim.x) {
      const int l = idx / (NRC_W * NRC_W), rem = idx % (NRC_W * NRC_W), o = rem / NRC_W, i = rem % NRC_W;
      t[(l * NRC_W + i) * NRC_LD + o] = g[idx];
    }
    unsigned short* th = t + NRC_HIDDEN * NRC_W * NRC_LD;  // head^T: [i][24], o < 16 used
    for (int idx = threadIdx.x; idx < NRC_W * 16; idx += blockDim.x) {
      const int i = idx / 16, o = idx % 16;
      th[i * 24 + o] = o < NRC_OUT ? g[NRC_HIDDEN * NRC_W * NRC_W + o * NRC_W + i] : (unsigned short)0;
    }
  }
}

// Encode 16 records (rows) of a warp tile into padded shared rows (BF16): lanes
// 0..15 write words 0..17 (position) of rows 0..15, lanes 16..31 words 18..31.
__device__ __forceinline__ void encode_tile(const float* __restrict__ raw, long long row0, long long n,
                                            const float* lo, const float* inv_ext, __nv_bfloat16* tile) {
  const int lane = threadIdx.x & 31;
  const int r = lane & 15, half = lane >> 4;
  const long long rec = row0 + r;
  uint32_t* dst = reinterpret_cast<uint32_t*>(tile + r * NRC_LD);
  if (rec < n) {
    float rr[NRC_RAW];
#pragma unroll
    for (int k = 0; k < NRC_RAW; ++k) rr[k] = raw[rec * NRC_RAW + k];
    if (half == 0)
      nrc_encode_position(rr, lo, inv_ext, dst);
    else
      nrc_encode_direction(rr, dst + 18);
  } else {
    const int m0 = half ? 18 : 0, m1 = half ? 32 : 18;
    for (int m = m0; m < m1; ++m) dst[m] = 0u;
  }
}

// A fragments of the four 16-wide k-tiles of a 16x64 BF16 tile in shared memory.
__device__ __forceinline__ void load_a_frags(uint32_t (&A)[4][4], const __nv_bfloat16* tile) {
  const int lane = threadIdx.x & 31;
  const int row = (lane & 7) + 8 * ((lane >> 3) & 1);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) ldmatrix_x4(A[kk], tile + row * NRC_LD + 16 * kk + 8 * (lane >> 4));
}

// One 64->64 layer: C[j] (n-tile j) = A * W_l^T with W_l in padded shared rows [o][i].
__device__ __forceinline__ void layer64(float (&C)[8][4], const uint32_t (&A)[4][4], const __nv_bfloat16* Wl) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* w = reinterpret_cast<const uint32_t*>(Wl);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int base = ((8 * j + g) * NRC_LD + 16 * kk + 2 * t) >> 1;
      mma_bf16(C[j], A[kk], w[base], w[base + 4]);
    }
  }
}

// Activations of the next layer as A fragments (ReLU applied), from C fragments.
__device__ __forceinline__ void relu_to_a(uint32_t (&A)[4][4], const float (&C)[8][4]) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    A[kk][0] = pack_bf16(fmaxf(C[2 * kk][0], 0.f), fmaxf(C[2 * kk][1], 0.f));
    A[kk][1] = pack_bf16(fmaxf(C[2 * kk][2], 0.f), fmaxf(C[2 * kk][3], 0.f));
    A[kk][2] = pack_bf16(fmaxf(C[2 * kk + 1][0], 0.f), fmaxf(C[2 * kk + 1][1], 0.f));
    A[kk][3] = pack_bf16(fmaxf(C[2 * kk + 1][2], 0.f), fmaxf(C[2 * kk + 1][3], 0.f));
  }
}

// Store A fragments (a 16x64 BF16 tile) to padded shared rows.
__device__ __forceinline__ void store_a_frags(const uint32_t (&A)[4][4], __nv_bfloat16* tile) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t* s = reinterpret_cast<uint32_t*>(tile);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    s[(g * NRC_LD + 16 * kk + 2 * t) >> 1] = A[kk][0];
    s[((g + 8) * NRC_LD + 16 * kk + 2 * t) >> 1] = A[kk][1];
    s[(g * NRC_LD + 16 * kk + 8 + 2 * t) >> 1] = A[kk][2];
    s[((g + 8) * NRC_LD + 16 * kk + 8 + 2 * t) >> 1] = A[kk][3];
  }
}

// Copy a 16x64 padded shared tile to global rows [row0 .. row0+15] of a [n][64] BF16 array.
__device__ __forceinline__ void tile_to_global(const __nv_bfloat16* tile, __nv_bfloat16* dst, long long row0,
                                               long long n) {
  const int lane = threadIdx.x & 31;
  for (int idx = lane; idx < 16 * 32; idx += 32) {
    const int r = idx >> 5, c2 = idx & 31;
    if (row0 + r < n)
      reinterpret_cast<uint32_t*>(dst + (row0 + r) * NRC_W)[c2] =
          reinterpret_cast<const uint32_t*>(tile + r * NRC_LD)[c2];
  }
}

// Head: 64 -> 3 (one n-tile of 8, outputs 3..7 are zero weights).
__device__ __forceinline__ void head(float (&y)[4], const uint32_t (&A)[4][4], const __nv_bfloat16* W5) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* w = reinterpret_cast<const uint32_t*>(W5);
  y[0] = y[1] = y[2] = y[3] = 0.0f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int base = (g * NRC_LD + 16 * kk + 2 * t) >> 1;
    mma_bf16(y, A[kk], w[base], w[base + 4]);
  }
}

// ---------------------------------------------------------------- inference
// out[r][c] = MLP(encode(raw[r])).
__global__ void __launch_bounds__(128) nrc_infer_kernel(const float* __restrict__ raw, long long n, NrcBox box,
                                                        const __nv_bfloat16* __restrict__ W, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char nrc_smem[];
  __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(nrc_smem);
  __nv_bfloat16* tiles = Ws + NrcSmem::W_ELEMS;
  load_weights_smem(W, Ws, false);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* tile = tiles + warp * 16 * NRC_LD;
  const long long n_tiles = (n + 15) / 16;
  for (long long tl = (long long)blockIdx.x * 4 + warp; tl < n_tiles; tl += (long long)gridDim.x * 4) {
    const long long row0 = tl * 16;
    encode_tile(raw, row0, n, box.lo, box.inv_ext, tile);
    __syncwarp();
    uint32_t A[4][4];
    load_a_frags(A, tile);
    float C[8][4];
#pragma unroll 1
    for (int l = 0; l < NRC_HIDDEN; ++l) {
      layer64(C, A, Ws + l * NRC_W * NRC_LD);
      relu_to_a(A, C);
    }
    float y[4];
    head(y, A, Ws + NRC_HIDDEN * NRC_W * NRC_LD);
    if (t < 2) {
      const int c0 = 2 * t;
      if (row0 + g < n) {
        out[(row0 + g) * 3 + c0] = y[0];
        if (c0 + 1 < 3) out[(row0 + g) * 3 + c0 + 1] = y[1];
      }
      if (row0 + g + 8 < n) {
        out[(row0 + g + 8) * 3 + c0] = y[2];
        if (c0 + 1 < 3) out[(row0 + g + 8) * 3 + c0 + 1] = y[3];
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- training: forward + backward deltas
// For a batch of n records: X[l] (inputs of layer l, l = 0..5, BF16 [n][64]) and the
// deltas dZ[l] at each layer's output (l = 0..4: [n][64]; head: [n][64] with
// columns 0..2 used) are written for the weight-gradient kernel; the loss
// (relative L2, mean over the batch) is accumulated into *loss.
__global__ void __launch_bounds__(128) nrc_train_fb_kernel(const float* __restrict__ raw,
                                                           const float* __restrict__ target, long long n, NrcBox box,
                                                           const __nv_bfloat16* __restrict__ W,
                                                           __nv_bfloat16* __restrict__ X,
                                                           __nv_bfloat16* __restrict__ dZ, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char nrc_smem[];
  __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(nrc_smem);
  __nv_bfloat16* WTs = Ws + NrcSmem::W_ELEMS;
  __nv_bfloat16* W5T = WTs + NRC_HIDDEN * NRC_W * NRC_LD;  // [64][24]
  __nv_bfloat16* tiles = W5T + NRC_W * 24;                 // per warp: 6 tiles of 16 x NRC_LD
  load_weights_smem(W, Ws, true);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* wt = tiles + warp * 6 * 16 * NRC_LD;
  const long long n_tiles = (n + 15) / 16;
  const float inv_n = 1.0f / (float)n;
  float loss_acc = 0.0f;
  const long long plane = n * NRC_W;
  for (long long tl = (long long)blockIdx.x * 4 + warp; tl < n_tiles; tl += (long long)gridDim.x * 4) {
    const long long row0 = tl * 16;
    encode_tile(raw, row0, n, box.lo, box.inv_ext, wt);
    __syncwarp();
    uint32_t A[4][4];
    load_a_frags(A, wt);
    tile_to_global(wt, X, row0, n);
    float C[8][4];
#pragma unroll 1
    for (int l = 0; l < NRC_HIDDEN; ++l) {
      layer64(C, A, Ws + l * NRC_W * NRC_LD);
      relu_to_a(A, C);
      store_a_frags(A, wt + (l + 1) * 16 * NRC_LD);
      __syncwarp();
      tile_to_global(wt + (l + 1) * 16 * NRC_LD, X + (l + 1) * plane, row0, n);
    }
    float y[4];
    head(y, A, Ws + NRC_HIDDEN * NRC_W * NRC_LD);
    // loss gradient at the outputs (columns 2t, 2t+1 of rows g, g+8)
    float dy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 2 * t + (q & 1);
      const long long rec = row0 + g + ((q & 2) ? 8 : 0);
      if (c < NRC_OUT && rec < n) {
        const float tv = target[rec * 3 + c];
        const float den = y[q] * y[q] + 0.01f;
        const float diff = y[q] - tv;
        loss_acc += diff * diff / den * inv_n;
        dy[q] = 2.0f * diff / den * inv_n;
      }
    }
    // head delta as A fragments (k-tile 0 = outputs 0..15, only 0..2 non-zero);
    // tile 0 (the encoding, already written out) is reused as staging
    uint32_t D[4][4] = {{pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), 0u, 0u},
                        {0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
    store_a_frags(D, wt);
    __syncwarp();
    tile_to_global(wt, dZ + NRC_HIDDEN * plane, row0, n);
    // dX5 = dy * W5 : B[k = o][n = i] = W5T[i][o]
    {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W5T);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.0f;
        const int base = ((8 * j + g) * 24 + 2 * t) >> 1;
        mma_bf16(C[j], D[0], w[base], w[base + 4]);
      }
    }
    // layers 4 .. 0: dZ_l = dX_{l+1} * relu'(X_{l+1}); store; dX_l = dZ_l * W_l
#pragma unroll 1
    for (int l = NRC_HIDDEN - 1; l >= 0; --l) {
      const uint32_t* xs = reinterpret_cast<const uint32_t*>(wt + (l + 1) * 16 * NRC_LD);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * kk + h;
          const uint32_t x_lo = xs[(g * NRC_LD + 8 * j + 2 * t) >> 1];
          const uint32_t x_hi = xs[((g + 8) * NRC_LD + 8 * j + 2 * t) >> 1];
          const float d0 = bf16_lo(x_lo) > 0.f ? C[j][0] : 0.f;
          const float d1 = bf16_hi(x_lo) > 0.f ? C[j][1] : 0.f;
          const float d2 = bf16_lo(x_hi) > 0.f ? C[j][2] : 0.f;
          const float d3 = bf16_hi(x_hi) > 0.f ? C[j][3] : 0.f;
          D[kk][2 * h] = pack_bf16(d0, d1);
          D[kk][2 * h + 1] = pack_bf16(d2, d3);
        }
      }
      store_a_frags(D, wt);
      __syncwarp();
      tile_to_global(wt, dZ + l * plane, row0, n);
      if (l == 0) break;
      const uint32_t* w = reinterpret_cast<const uint32_t*>(WTs + l * NRC_W * NRC_LD);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int base = ((8 * j + g) * NRC_LD + 16 * kk + 2 * t) >> 1;
          mma_bf16(C[j], D[kk], w[base], w[base + 4]);
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
  if (lane == 0 && loss_acc != 0.0f) atomicAdd(loss, loss_acc);
}

// ---------------------------------------------------------------- training: weight gradients
// dW_l[o][i] += sum_b dZ_l[b][o] * X_l[b][i] (split-K over blocks; blockIdx.y = layer,
// the head is layer 5 with o < 3).  Each block stages 64 records of dZ_l and X_l in
// shared memory; warp w owns output rows o in [16w, 16w+16).
__global__ void __launch_bounds__(128) nrc_wgrad_kernel(const __nv_bfloat16* __restrict__ X,
                                                        const __nv_bfloat16* __restrict__ dZ, long long n,
                                                        long long chunk, float* __restrict__ dW) {
  __shared__ __align__(16) __nv_bfloat16 sz[64 * NRC_LD];
  __shared__ __align__(16) __nv_bfloat16 sx[64 * NRC_LD];
  const int l = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long plane = n * NRC_W;
  const __nv_bfloat16* Xl = X + l * plane;
  const __nv_bfloat16* Zl = dZ + l * plane;
  const long long b_begin = (long long)blockIdx.x * chunk;
  const long long b_end = b_begin + chunk < n ? b_begin + chunk : n;
  const int m0 = 16 * warp;
  const bool active = (l < NRC_HIDDEN) || warp == 0;
  float C[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) C[j][0] = C[j][1] = C[j][2] = C[j][3] = 0.0f;
  for (long long b0 = b_begin; b0 < b_end; b0 += 64) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * 32; idx += blockDim.x) {
      const int r = idx >> 5, c2 = idx & 31;
      uint32_t zv = 0u, xv = 0u;
      if (b0 + r < b_end) {
        zv = reinterpret_cast<const uint32_t*>(Zl + (b0 + r) * NRC_W)[c2];
        xv = reinterpret_cast<const uint32_t*>(Xl + (b0 + r) * NRC_W)[c2];
      }
      reinterpret_cast<uint32_t*>(sz + r * NRC_LD)[c2] = zv;
      reinterpret_cast<uint32_t*>(sx + r * NRC_LD)[c2] = xv;
    }
    __syncthreads();
    if (!active) continue;
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 16) {
      uint32_t A[4];
      {
        const int q = lane >> 3;
        const int br = k0 + 8 * (q >> 1) + (lane & 7);
        const int oc = m0 + 8 * (q & 1);
        ldmatrix_x4_trans(A, sz + br * NRC_LD + oc);
      }
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        uint32_t B[4];
        const int q = lane >> 3;
        const int br = k0 + 8 * (q & 1) + (lane & 7);
        const int ic = 8 * (j + (q >> 1));
        ldmatrix_x4_trans(B, sx + br * NRC_LD + ic);
        mma_bf16(C[j], A, B[0], B[1]);
        mma_bf16(C[j + 1], A, B[2], B[3]);
      }
    }
  }
  if (!active) return;
  float* dWl = dW + (size_t)l * NRC_W * NRC_W;
  const int o_lim = l < NRC_HIDDEN ? NRC_W : NRC_OUT;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i0 = 8 * j + 2 * t;
    const int oa = m0 + g, ob = m0 + g + 8;
    if (oa < o_lim) {
      atomicAdd(&dWl[oa * NRC_W + i0], C[j][0]);
      atomicAdd(&dWl[oa * NRC_W + i0 + 1], C[j][1]);
    }
    if (ob < o_lim) {
      atomicAdd(&dWl[ob * NRC_W + i0], C[j][2]);
      atomicAdd(&dWl[ob * NRC_W + i0 + 1], C[j][3]);
    }
  }
}

// ---------------------------------------------------------------- Adam
// One Adam step of every parameter; with ema > 0 also the exponential moving
// average of the weights (Polyak averaging) and its BF16 copy, which queries use.
__global__ void nrc_adam_kernel(float* __restrict__ W32, float* __restrict__ dW, float* __restrict__ m,
                                float* __restrict__ v, __nv_bfloat16* __restrict__ Wb, float lr, float b1, float b2,
                                float eps, float c1, float c2, float* __restrict__ Wavg,
                                __nv_bfloat16* __restrict__ Wq, float ema) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NRC_PARAMS) return;
  const float gr = dW[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gr;
  const float vi = b2 * v[i] + (1.0f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  const float w = W32[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  W32[i] = w;
  Wb[i] = __float2bfloat16_rn(w);
  dW[i] = 0.0f;
  if (ema > 0.0f) {
    const float a = ema * Wavg[i] + (1.0f - ema) * w;
    Wavg[i] = a;
    Wq[i] = __float2bfloat16_rn(a);
  }
}

__global__ void nrc_to_bf16_kernel(const float* __restrict__ W32, __nv_bfloat16* __restrict__ Wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NRC_PARAMS) Wb[i] = __float2bfloat16_rn(W32[i]);
}

}  // namespace ptgb

// ============================================================================ C ABI
using namespace ptgb;

struct pt_cache {
  pt_cache_desc desc;
  NrcBox box;
  float* W32 = nullptr;     // master weights
  float* m = nullptr;
  float* v = nullptr;
  float* dW = nullptr;
  __nv_bfloat16* Wb = nullptr;  // [NRC_HIDDEN*64*64 + 8*64]
  float* Wavg = nullptr;        // moving average of W32 (desc.ema > 0)
  __nv_bfloat16* Wq = nullptr;  // its BF16 copy: the weights queries use when desc.ema > 0
  __nv_bfloat16* X = nullptr;   // [6][batch][64]
  __nv_bfloat16* dZ = nullptr;  // [6][batch][64]
  float* loss = nullptr;        // [1]
  float* q_raw = nullptr;       // queries [max_queries][10]
  float* q_beta = nullptr;      // [max_queries][3]
  float* q_rgb = nullptr;       // [max_queries][3]
  float* r_raw = nullptr;       // training records [max_records][10]
  float* r_aux = nullptr;       // [max_records][8]: beta(3), L_before(3), path id (as bits), pad
  float* r_target = nullptr;    // [max_records][3]
  float* path_L = nullptr;      // [max_paths][3] final radiance of training paths
  unsigned* r_count = nullptr;  // [2] records written, paths written
  int* status = nullptr;        // [1] device-side error of the tensor-core kernels
  int engine = PT_CACHE_TCGEN05;
  unsigned wait_limit = PT_CACHE_WAIT_LIMIT_DEFAULT;  // per-step bounded-wait polls of the tensor-core kernels
  int step = 0;
};

namespace {

constexpr size_t kInferSmem = (size_t)NrcSmem::W_ELEMS * 2 + 4 * 16 * NRC_LD * 2;
constexpr size_t kTrainSmem = (size_t)NrcSmem::W_ELEMS * 2 + (size_t)NRC_HIDDEN * NRC_W * NRC_LD * 2 +
                              NRC_W * 24 * 2 + 4 * 6 * 16 * NRC_LD * 2;

void cache_free(pt_cache* c) {
  void* ptrs[] = {c->W32, c->m, c->v, c->dW, c->Wb, c->Wavg, c->Wq, c->X, c->dZ, c->loss, c->q_raw, c->q_beta, c->q_rgb,
                  c->r_raw, c->r_aux, c->r_target, c->path_L, c->r_count, c->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

bool smem_opt_in() {
  static int done = 0;
  if (!done) {
    if (cudaFuncSetAttribute(nrc_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(nrc_train_fb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem) !=
            cudaSuccess)
      return false;
    done = 1;
  }
  return true;
}

// Library default initialisation: uniform +-sqrt(6 / fan_in) (He-style for ReLU)
// from a 64-bit LCG stream seeded by desc.seed.
void default_init(std::vector<float>& w, uint64_t seed) {
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  float a = std::sqrt(6.0f / NRC_W);
  for (auto& x : w) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    float u = (float)((s >> 40) & 0xffffff) / 16777216.0f;
    x = (2.0f * u - 1.0f) * a;
  }
}

}  // namespace

extern "C" int pt_cache_create(const pt_cache_desc* d, pt_cache** out) {
  if (!d || !out) return PT_ERR_ARG;
  *out = nullptr;
  if (d->batch <= 0 || d->batch % 64 || d->max_queries < 0 || d->max_records < 0 || d->max_paths < 0)
    return PT_ERR_ARG;
  if (!(d->ema >= 0.0f && d->ema < 1.0f)) return PT_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (!(d->box_hi[k] > d->box_lo[k])) return PT_ERR_ARG;
  if (!smem_opt_in()) return PT_ERR_CUDA;
  pt_cache* c = new (std::nothrow) pt_cache();
  if (!c) return PT_ERR_OOM;
  c->desc = *d;
  for (int k = 0; k < 3; ++k) {
    c->box.lo[k] = d->box_lo[k];
    c->box.inv_ext[k] = 1.0f / (d->box_hi[k] - d->box_lo[k]);
  }
  const size_t nb = (size_t)NRC_HIDDEN * NRC_W * NRC_W + 8 * NRC_W;
  const size_t act = (size_t)(NRC_HIDDEN + 1) * d->batch * NRC_W;
  bool ok = cudaMalloc(&c->W32, NRC_PARAMS * 4) == cudaSuccess && cudaMalloc(&c->m, NRC_PARAMS * 4) == cudaSuccess &&
            cudaMalloc(&c->v, NRC_PARAMS * 4) == cudaSuccess && cudaMalloc(&c->dW, NRC_PARAMS * 4) == cudaSuccess &&
            cudaMalloc(&c->Wb, nb * 2) == cudaSuccess && cudaMalloc(&c->Wavg, NRC_PARAMS * 4) == cudaSuccess &&
            cudaMalloc(&c->Wq, nb * 2) == cudaSuccess && cudaMalloc(&c->X, act * 2) == cudaSuccess &&
            cudaMalloc(&c->dZ, act * 2) == cudaSuccess && cudaMalloc(&c->loss, 4) == cudaSuccess &&
            cudaMalloc(&c->r_count, 8) == cudaSuccess && cudaMalloc(&c->status, 4) == cudaSuccess;
  if (ok && d->max_queries > 0)
    ok = cudaMalloc(&c->q_raw, (size_t)d->max_queries * NRC_RAW * 4) == cudaSuccess &&
         cudaMalloc(&c->q_beta, (size_t)d->max_queries * 12) == cudaSuccess &&
         cudaMalloc(&c->q_rgb, (size_t)d->max_queries * 12) == cudaSuccess;
  if (ok && d->max_records > 0)
    ok = cudaMalloc(&c->r_raw, (size_t)d->max_records * NRC_RAW * 4) == cudaSuccess &&
         cudaMalloc(&c->r_aux, (size_t)d->max_records * 32) == cudaSuccess &&
         cudaMalloc(&c->r_target, (size_t)d->max_records * 12) == cudaSuccess;
  if (ok && d->max_paths > 0) ok = cudaMalloc(&c->path_L, (size_t)d->max_paths * 12) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cache_free(c);
    delete c;
    return PT_ERR_OOM;
  }
  std::vector<float> w(NRC_PARAMS);
  if (d->init_weights) std::memcpy(w.data(), d->init_weights, sizeof(float) * NRC_PARAMS);
  else default_init(w, d->seed);
  ok = cudaMemcpy(c->W32, w.data(), NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(c->m, 0, NRC_PARAMS * 4) == cudaSuccess && cudaMemset(c->v, 0, NRC_PARAMS * 4) == cudaSuccess &&
       cudaMemset(c->dW, 0, NRC_PARAMS * 4) == cudaSuccess && cudaMemset(c->Wb, 0, nb * 2) == cudaSuccess &&
       cudaMemset(c->Wq, 0, nb * 2) == cudaSuccess &&
       cudaMemcpy(c->Wavg, w.data(), NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(c->loss, 0, 4) == cudaSuccess && cudaMemset(c->r_count, 0, 8) == cudaSuccess &&
       cudaMemset(c->status, 0, 4) == cudaSuccess;
  if (ok) {
    nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->W32, c->Wb);
    nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->Wavg, c->Wq);
    ok = cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    cache_free(c);
    delete c;
    return PT_ERR_CUDA;
  }
  *out = c;
  return PT_OK;
}

extern "C" void pt_cache_destroy(pt_cache* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cache_free(c);
  delete c;
}

extern "C" int pt_cache_get_weights(pt_cache* c, float* host_out) {
  if (!c || !host_out) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  return cudaMemcpy(host_out, c->W32, NRC_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_set_weights(pt_cache* c, const float* host_in) {
  if (!c || !host_in) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  bool ok = cudaMemcpy(c->W32, host_in, NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(c->m, 0, NRC_PARAMS * 4) == cudaSuccess && cudaMemset(c->v, 0, NRC_PARAMS * 4) == cudaSuccess &&
            cudaMemset(c->dW, 0, NRC_PARAMS * 4) == cudaSuccess;
  if (!ok || cudaMemcpy(c->Wavg, host_in, NRC_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess) return PT_ERR_CUDA;
  c->step = 0;
  nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->W32, c->Wb);
  nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->Wavg, c->Wq);
  return cudaDeviceSynchronize() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

namespace ptgb {
int cache_infer(pt_cache* c, const float* raw, float* rgb, long long n, cudaStream_t st) {
  if (n <= 0) return PT_OK;
  const __nv_bfloat16* Wuse = c->desc.ema > 0.0f ? c->Wq : c->Wb;
  if (c->engine == PT_CACHE_TCGEN05) return cache_infer_tc(raw, rgb, n, c->box, Wuse, c->status, c->wait_limit, st);
  const long long tiles = (n + 15) / 16;
  long long grid = (tiles + 3) / 4;
  if (grid > 152 * 8) grid = 152 * 8;
  nrc_infer_kernel<<<(unsigned)grid, 128, kInferSmem, st>>>(raw, n, c->box, Wuse, rgb);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

// `steps` optimisation steps over consecutive batches of the n records.
int cache_optimise(pt_cache* c, const float* raw, const float* target, long long n, int steps, cudaStream_t st) {
  const long long B = c->desc.batch;
  if (n <= 0 || steps <= 0) return PT_OK;
  for (int s = 0; s < steps; ++s) {
    const long long off = (long long)(((long long)s * B) % (n > B ? n - B + 1 : 1));
    const long long nb = n < B ? n : B;
    const long long tiles = (nb + 15) / 16;
    long long grid = (tiles + 3) / 4;
    if (grid > 152 * 4) grid = 152 * 4;
    cudaMemsetAsync(c->loss, 0, 4, st);
    if (c->engine == PT_CACHE_TCGEN05) {
      const int rc = cache_train_fb_tc(raw + off * NRC_RAW, target + off * 3, nb, c->box, c->Wb, c->X, c->dZ, c->loss,
                                       c->status, c->wait_limit, st);
      if (rc != PT_OK) return rc;
    } else {
      nrc_train_fb_kernel<<<(unsigned)grid, 128, kTrainSmem, st>>>(raw + off * NRC_RAW, target + off * 3, nb, c->box,
                                                                   c->Wb, c->X, c->dZ, c->loss);
    }
    const long long chunk = 512;
    if (c->engine == PT_CACHE_TCGEN05) {
      const int rc = cache_wgrad_tc(c->X, c->dZ, nb, chunk, c->dW, c->status, c->wait_limit, st);
      if (rc != PT_OK) return rc;
    } else {
      dim3 g2((unsigned)((nb + chunk - 1) / chunk), NRC_HIDDEN + 1);
      nrc_wgrad_kernel<<<g2, 128, 0, st>>>(c->X, c->dZ, nb, chunk, c->dW);
    }
    c->step += 1;
    const pt_cache_desc& d = c->desc;
    const float c1 = 1.0f - std::pow(d.beta1, (float)c->step), c2 = 1.0f - std::pow(d.beta2, (float)c->step);
    nrc_adam_kernel<<<(NRC_PARAMS + 255) / 256, 256, 0, st>>>(c->W32, c->dW, c->m, c->v, c->Wb, d.lr, d.beta1,
                                                              d.beta2, d.eps, c1, c2, c->Wavg, c->Wq, d.ema);
  }
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
}  // namespace ptgb

namespace ptgb {
CacheBuffers cache_buffers(pt_cache* c) {
  CacheBuffers b;
  b.q_raw = c->q_raw;
  b.q_beta = c->q_beta;
  b.q_rgb = c->q_rgb;
  b.r_raw = c->r_raw;
  b.r_aux = c->r_aux;
  b.r_target = c->r_target;
  b.path_L = c->path_L;
  b.r_count = c->r_count;
  b.max_queries = c->desc.max_queries;
  b.max_records = c->desc.max_records;
  b.max_paths = c->desc.max_paths;
  return b;
}
}  // namespace ptgb

extern "C" int pt_cache_query(pt_cache* c, const float* raw, float* rgb, int n, void* stream) {
  if (!c || n < 0 || (n > 0 && (!raw || !rgb))) return PT_ERR_ARG;
  return cache_infer(c, raw, rgb, n, (cudaStream_t)stream);
}

// The BF16 features both inference engines feed to the first layer: one thread per
// record, words[i] = nrc_encode_packed(raw[i]).
__global__ void __launch_bounds__(256) nrc_encode_kernel(const float* __restrict__ raw, long long n, NrcBox box,
                                                         uint4* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float rr[NRC_RAW];
#pragma unroll
  for (int k = 0; k < NRC_RAW; ++k) rr[k] = raw[i * NRC_RAW + k];
  uint32_t w[32];
  nrc_encode_packed(rr, box.lo, box.inv_ext, true, w);
#pragma unroll
  for (int c = 0; c < 8; ++c) out[i * 8 + c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
}

extern "C" int pt_cache_encode(pt_cache* c, const float* raw, uint16_t* features, int n, void* stream) {
  if (!c || n < 0 || (n > 0 && (!raw || !features))) return PT_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(features) & 15u) != 0) return PT_ERR_ARG;
  if (n == 0) return PT_OK;
  nrc_encode_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(raw, n, c->box,
                                                                                  reinterpret_cast<uint4*>(features));
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_set_engine(pt_cache* c, int engine) {
  if (!c || (engine != PT_CACHE_TCGEN05 && engine != PT_CACHE_MMA_SYNC)) return PT_ERR_ARG;
  c->engine = engine;
  return PT_OK;
}

extern "C" int pt_cache_get_state(pt_cache* c, float* w, float* m, float* v, int32_t* step) {
  if (!c || !w || !m || !v || !step) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  const bool ok = cudaMemcpy(w, c->W32, NRC_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
                  cudaMemcpy(m, c->m, NRC_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
                  cudaMemcpy(v, c->v, NRC_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (!ok) return PT_ERR_CUDA;
  *step = c->step;
  return PT_OK;
}

extern "C" int pt_cache_set_state(pt_cache* c, const float* w, const float* m, const float* v, int32_t step) {
  if (!c || !w || !m || !v || step < 0) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  const bool ok = cudaMemcpy(c->W32, w, NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(c->m, m, NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(c->v, v, NRC_PARAMS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemset(c->dW, 0, NRC_PARAMS * 4) == cudaSuccess;
  if (!ok) return PT_ERR_CUDA;
  c->step = step;
  nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->W32, c->Wb);
  return cudaDeviceSynchronize() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_get_average(pt_cache* c, float* host_out) {
  if (!c || !host_out) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  return cudaMemcpy(host_out, c->Wavg, NRC_PARAMS * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_set_average(pt_cache* c, const float* host_in) {
  if (!c || !host_in) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(c->Wavg, host_in, NRC_PARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return PT_ERR_CUDA;
  nrc_to_bf16_kernel<<<(NRC_PARAMS + 255) / 256, 256>>>(c->Wavg, c->Wq);
  return cudaDeviceSynchronize() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_set_wait_limit(pt_cache* c, uint32_t limit) {
  if (!c) return PT_ERR_ARG;
  c->wait_limit = limit;
  return PT_OK;
}

extern "C" int pt_cache_status(pt_cache* c, void* stream, int* out) {
  if (!c || !out) return PT_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PT_ERR_CUDA;
  if (cudaMemcpy(out, c->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PT_ERR_CUDA;
  return cudaMemset(c->status, 0, 4) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_train_records(pt_cache* c, const float* raw, const float* target, int n, int steps,
                                      void* stream) {
  if (!c || n < 0 || steps < 0 || (n > 0 && (!raw || !target))) return PT_ERR_ARG;
  return cache_optimise(c, raw, target, n, steps, (cudaStream_t)stream);
}

extern "C" int pt_cache_last_loss(pt_cache* c, void* stream, float* out) {
  if (!c || !out) return PT_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PT_ERR_CUDA;
  return cudaMemcpy(out, c->loss, 4, cudaMemcpyDeviceToHost) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

extern "C" int pt_cache_read_records(pt_cache* c, int cap, float* raw, float* target, int* meta, int* n_out) {
  if (!c || cap < 0 || !n_out) return PT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
  unsigned count = 0;
  if (cudaMemcpy(&count, c->r_count, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return PT_ERR_CUDA;
  long long n = count;
  if (n > c->desc.max_records) n = c->desc.max_records;
  if (n > cap) n = cap;
  *n_out = (int)n;
  if (n == 0) return PT_OK;
  std::vector<float> aux((size_t)n * 8);
  bool ok = (!raw || cudaMemcpy(raw, c->r_raw, (size_t)n * 40, cudaMemcpyDeviceToHost) == cudaSuccess) &&
            (!target || cudaMemcpy(target, c->r_target, (size_t)n * 12, cudaMemcpyDeviceToHost) == cudaSuccess) &&
            cudaMemcpy(aux.data(), c->r_aux, (size_t)n * 32, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (!ok) return PT_ERR_CUDA;
  if (meta)
    for (long long i = 0; i < n; ++i) {
      std::memcpy(&meta[2 * i], &aux[i * 8 + 6], 4);
      std::memcpy(&meta[2 * i + 1], &aux[i * 8 + 7], 4);
    }
  return PT_OK;
}
