// Radiance-cache MLP inference on the 5th-generation tensor cores (tcgen05):
// the MMAs are issued by one thread with operands in shared memory (UMMA
// descriptors, K-major, no swizzle), accumulators live in tensor memory and are
// read back with tcgen05.ld for the ReLU / BF16 epilogue, which writes the next
// layer's operand tile.  128 queries per tile (M = 128), 64-wide layers (N = 64,
// K = 64 as four K = 16 steps), a 16-wide head (3 outputs used).  Same network
// encoding and BF16 rounding points as the mma.sync kernel in pt_nrc.cu.
#include <cuda_bf16.h>

#include "pt_internal.h"
#include "pt_nrc.cuh"

namespace ptgb {
namespace {

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on the barrier phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned limit) {
  const uint32_t a = smem_addr(bar);
  for (unsigned i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading-dimension byte offset
// (between core matrices along K), stride byte offset (between 8-row groups),
// the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape), waited on.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n tcgen05.wait::ld.sync.aligned;\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// BF16 pair (lo in the low half) of max(x, 0): one convert with ReLU, the same bits
// as pack_bf16(fmaxf(lo, 0), fmaxf(hi, 0)) for finite inputs.
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// ---------------------------------------------------------------- operand layout
// K-major, no swizzle, K = 64: 8x8 core matrices of 8 rows x 16 bytes, the eight
// core matrices of an 8-row group adjacent along K (128 B apart), 8-row groups
// 1024 B apart.  A K = 16 step covers two core matrices along K (256 B).
constexpr uint32_t kLBO = 128, kSBO = 1024;
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// One CTA per SM, kGroups independent groups of 128 threads.  A group owns one
// 128-query activation tile, 64 TMEM columns and an mbarrier, and runs its own
// tiles through the layer chain; while one group's tile sits in the tensor core
// the other groups run their epilogues and encodings.  The weights are loaded
// into shared memory once per CTA.
constexpr int kGroups = 8;
constexpr uint32_t kSmW = 0, kSmH = 5 * 8192, kSmX = kSmH + 2048;
constexpr uint32_t kRawTile = 128 * NRC_RAW * 4;  // one tile's raw records: 5120 bytes
constexpr uint32_t kSmRaw = kSmX + kGroups * 16384;
constexpr uint32_t kSmBar = kSmRaw + kGroups * kRawTile, kSmSlot = kSmBar + 8 * kGroups;
constexpr uint32_t kTcSmem = kSmSlot + 8 + 1024;  // + alignment slack
constexpr uint32_t kTmemCols = 64 * kGroups;      // 512: the whole tensor memory of the SM
// Bounded waits: per MMA step `limit` polls (the cache's wait limit, by default
// kWaitLimit; a smaller one is a failure-injection hook), and always kWaitLimit
// for the final wait (on the parity of the wait that gave up) that lets an MMA in
// flight finish before TMEM is released.
constexpr unsigned kWaitLimit = PT_CACHE_WAIT_LIMIT_DEFAULT;

// Barrier over the 128 threads of group g (named barrier 1 + g), AND of `pred`.
__device__ __forceinline__ bool group_sync_and(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.and.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(1 + g)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("barrier.cta.sync %0, 128;" ::"r"(1 + g) : "memory");
}

// Asynchronous 4-byte copies from global to shared memory (no registers held while
// they are in flight); a thread's copies are complete after cp_async_wait_all, and
// visible to the other threads after a barrier that follows it.
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Thread r's share of tile `tile`'s raw records into a group's staging buffer:
// floats r, r + 128, ..., r + 1152 of the tile's 1280 (each warp copies 128
// contiguous bytes at a time).  Floats past the end of the input are not copied;
// their rows are not live.
__device__ __forceinline__ void stage_raw(uint32_t stage_s, const float* raw, long long tile, long long n, int r) {
  const long long base = tile * (128LL * NRC_RAW), end = n * NRC_RAW;
#pragma unroll
  for (int j = 0; j < NRC_RAW; ++j) {
    const long long e = base + r + 128 * j;
    if (e < end) cp_async4(stage_s + 4u * (uint32_t)(r + 128 * j), raw + e);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(128 * kGroups, 1)
    nrc_infer_tc_kernel(const float* __restrict__ raw, long long n, NrcBox box, const __nv_bfloat16* __restrict__ W,
                        float* __restrict__ out, int* __restrict__ status, unsigned limit) {
  extern __shared__ unsigned char tc_smem_raw[];
  // 1024-byte aligned base for the operand tiles
  unsigned char* sm = tc_smem_raw + ((1024u - (smem_addr(tc_smem_raw) & 1023u)) & 1023u);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmSlot);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 7, r = tid & 127;  // group, row of the group's tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmBar) + g;
  unsigned char* X = sm + kSmX + g * 16384;

  // weights into the operand layout: layer l is B = W_l[o][i] (N = o, K = i)
  const unsigned short* gw = reinterpret_cast<const unsigned short*>(W);
  for (int idx = tid; idx < NRC_HIDDEN * NRC_W * NRC_W; idx += blockDim.x) {
    const int l = idx >> 12, o = (idx >> 6) & 63, i = idx & 63;
    *reinterpret_cast<unsigned short*>(sm + kSmW + l * 8192 + core_off(o, i)) = gw[idx];
  }
  for (int idx = tid; idx < 16 * NRC_W; idx += blockDim.x) {
    const int o = idx >> 6, i = idx & 63;
    *reinterpret_cast<unsigned short*>(sm + kSmH + core_off(o, i)) =
        o < NRC_OUT ? gw[NRC_HIDDEN * NRC_W * NRC_W + o * NRC_W + i] : (unsigned short)0;
  }
  // The group's raw records go through a staging buffer: each tile's are copied
  // while the previous tile runs through the layers.
  const float* stage = reinterpret_cast<const float*>(sm + kSmRaw + g * kRawTile);
  const uint32_t stage_s = smem_addr(stage);
  const long long n_tiles = (n + 127) / 128, stride = (long long)gridDim.x * kGroups;
  long long tile = (long long)blockIdx.x * kGroups + g;
  if (tile < n_tiles) stage_raw(stage_s, raw, tile, n, r);
  cp_async_wait_all();
  if (r == 0) mbar_init(bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot + 64u * g;  // this group's 64 columns
  const uint32_t x_s = smem_addr(X), w_s = smem_addr(sm + kSmW), h_s = smem_addr(sm + kSmH);
  const uint32_t t_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's 32 TMEM lanes
  uint32_t phase = 0, last = 0;  // last: parity of the latest wait
  bool ok = true;
  for (; tile < n_tiles && ok; tile += stride) {
    // ---- encode this thread's query (row r of the tile), from the staged records
    const long long row = tile * 128 + r;
    float rr[NRC_RAW];
#pragma unroll
    for (int k = 0; k < NRC_RAW; k += 2) {
      const float2 v = row < n ? reinterpret_cast<const float2*>(stage + r * NRC_RAW)[k >> 1] : make_float2(0.f, 0.f);
      rr[k] = v.x;
      rr[k + 1] = v.y;
    }
    {
      uint32_t w[32];
      nrc_encode_packed(rr, box.lo, box.inv_ext, row < n, w);
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
        *reinterpret_cast<uint4*>(X + core_off(r, 8 * c8)) =
            make_uint4(w[4 * c8], w[4 * c8 + 1], w[4 * c8 + 2], w[4 * c8 + 3]);
    }
    fence_async_smem();
    tc_fence_before();
    group_sync(g);
    // every thread of the group has read its record: stage the next tile's
    if (tile + stride < n_tiles) stage_raw(stage_s, raw, tile + stride, n, r);
    // ---- five hidden layers and the head
    for (int l = 0; l <= NRC_HIDDEN; ++l) {
      const bool head = l == NRC_HIDDEN;
      if (r == 0) {
        tc_fence_after();
        const uint32_t b_s = head ? h_s : w_s + (uint32_t)l * 8192u;
        const uint32_t idesc = head ? idesc_bf16(128, 16) : idesc_bf16(128, 64);
#pragma unroll
        for (int s = 0; s < 4; ++s)
          umma_bf16(tmem, umma_desc(x_s + 256u * s, kLBO, kSBO), umma_desc(b_s + 256u * s, kLBO, kSBO), idesc,
                    s > 0 ? 1u : 0u);
        umma_commit(bar);
      }
      // each thread waits for the commit itself (the warp takes the AND, so that the
      // warp-collective TMEM loads below run in all of its lanes or in none); the
      // group agrees on the outcome at the end of the layer
      const bool done = __all_sync(0xffffffffu, mbar_wait(bar, last = phase, limit));
      phase ^= 1u;
      tc_fence_after();
      if (!done) {
        // gave up: no TMEM read of an unfinished accumulator, outputs not written
      } else if (!head) {
        // ReLU + BF16 of this thread's row -> the next operand tile
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
          float v[16];
          tmem_ld16(t_lane + 16u * c16, v);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float* p = v + 8 * h;
            const uint4 q = make_uint4(pack_relu_bf16(p[0], p[1]), pack_relu_bf16(p[2], p[3]),
                                       pack_relu_bf16(p[4], p[5]), pack_relu_bf16(p[6], p[7]));
            *reinterpret_cast<uint4*>(X + core_off(r, 16 * c16 + 8 * h)) = q;
          }
        }
        fence_async_smem();
      } else {
        float v[16];
        tmem_ld16(t_lane, v);
        if (row < n) {
          out[row * 3] = v[0];
          out[row * 3 + 1] = v[1];
          out[row * 3 + 2] = v[2];
        }
        cp_async_wait_all();  // the next tile's records, visible to the group after the barrier
      }
      tc_fence_before();
      ok = group_sync_and(g, done);
      if (!ok) break;
    }
  }
  cp_async_wait_all();  // no copy in flight past a loop left early
  if (!ok) {
    if (r == 0) atomicCAS(status, 0, PT_ERR_TIMEOUT);
    // let an MMA still in flight finish before the tensor memory is released
    mbar_wait(bar, last, kWaitLimit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*slot), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------- training: forward + backward deltas
// The mma.sync training kernel's computation on tcgen05, group by group: per
// 128-record tile, the forward chain writes X_0..X_5 (BF16, [n][64] per layer),
// the head gives y, the relative-L2 loss and dy = 2 (y - t) / (y^2 + 0.01) / n
// (rounded to BF16, written to dZ_5 columns 0..2), then
//   dX_5 = dY Wh,  dZ_l = dX_{l+1} * [X_{l+1} > 0]  (BF16, written to dZ_l),
//   dX_l = dZ_l W_l  (l = 4 .. 1).
// The backward products use transposed weight tiles (B[n = i][k = o] = W[o][i]).
constexpr int kTrGroups = 4;
constexpr uint32_t kTrW = 0, kTrH = 40960, kTrWT = kTrH + 2048, kTrHT = kTrWT + 40960;
constexpr uint32_t kTrX = kTrHT + 2048;                        // per group: 128x64 operand tile
constexpr uint32_t kTrY = kTrX + kTrGroups * 16384;            // per group: 128x16 head-delta tile
constexpr uint32_t kTrBar = kTrY + kTrGroups * 4096, kTrSlot = kTrBar + 8 * kTrGroups;
constexpr uint32_t kTrSmem = kTrSlot + 8 + 1024;
constexpr uint32_t kTrCols = 64 * kTrGroups;

// K = 16 operand tile: two core matrices along K (128 B apart), 8-row groups 256 B apart.
__device__ __forceinline__ uint32_t core16_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Issue D = A B^T over K = 64 (four K = 16 steps), or one step for K = 16 tiles.
__device__ __forceinline__ void issue_k64(uint32_t d, uint32_t a_s, uint32_t b_s, uint32_t idesc, uint64_t* bar) {
  tc_fence_after();
#pragma unroll
  for (int s = 0; s < 4; ++s)
    umma_bf16(d, umma_desc(a_s + 256u * s, kLBO, kSBO), umma_desc(b_s + 256u * s, kLBO, kSBO), idesc,
              s > 0 ? 1u : 0u);
  umma_commit(bar);
}
__device__ __forceinline__ void issue_k16(uint32_t d, uint32_t a_s, uint32_t b_s, uint32_t idesc, uint64_t* bar) {
  tc_fence_after();
  umma_bf16(d, umma_desc(a_s, 128, 256), umma_desc(b_s, 128, 256), idesc, 0u);
  umma_commit(bar);
}

// Writes 8 BF16 values (one 16-byte chunk k8 of row `row`) to the operand tile and
// to the global row.
__device__ __forceinline__ void put_chunk(unsigned char* tile, int row, int k8, uint4 q, __nv_bfloat16* grow) {
  *reinterpret_cast<uint4*>(tile + core_off(row, 8 * k8)) = q;
  if (grow) reinterpret_cast<uint4*>(grow)[k8] = q;
}

__global__ void __launch_bounds__(128 * kTrGroups, 1)
    nrc_train_tc_kernel(const float* __restrict__ raw, const float* __restrict__ target, long long n, NrcBox box,
                        const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ X,
                        __nv_bfloat16* __restrict__ dZ, float* __restrict__ loss, int* __restrict__ status,
                        unsigned limit) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* sm = tc_smem_raw + ((1024u - (smem_addr(tc_smem_raw) & 1023u)) & 1023u);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kTrSlot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid >> 7, r = tid & 127;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTrBar) + g;
  unsigned char* Xt = sm + kTrX + g * 16384;
  unsigned char* Yt = sm + kTrY + g * 4096;

  // weights: forward tiles B[o][i] and transposed tiles B[i][o]; the head (3 rows used)
  const unsigned short* gw = reinterpret_cast<const unsigned short*>(W);
  for (int idx = tid; idx < NRC_HIDDEN * NRC_W * NRC_W; idx += blockDim.x) {
    const int l = idx >> 12, o = (idx >> 6) & 63, i = idx & 63;
    const unsigned short v = gw[idx];
    *reinterpret_cast<unsigned short*>(sm + kTrW + l * 8192 + core_off(o, i)) = v;
    *reinterpret_cast<unsigned short*>(sm + kTrWT + l * 8192 + core_off(i, o)) = v;
  }
  for (int idx = tid; idx < 16 * NRC_W; idx += blockDim.x) {
    const int o = idx >> 6, i = idx & 63;
    const unsigned short v = o < NRC_OUT ? gw[NRC_HIDDEN * NRC_W * NRC_W + o * NRC_W + i] : (unsigned short)0;
    *reinterpret_cast<unsigned short*>(sm + kTrH + core_off(o, i)) = v;   // [o(16)][i(64)]
    *reinterpret_cast<unsigned short*>(sm + kTrHT + core16_off(i, o)) = v;  // [i(64)][o(16)]
  }
  if (r == 0) mbar_init(bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(kTrCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot + 64u * g;
  const uint32_t x_s = smem_addr(Xt), y_s = smem_addr(Yt);
  const uint32_t w_s = smem_addr(sm + kTrW), h_s = smem_addr(sm + kTrH);
  const uint32_t wt_s = smem_addr(sm + kTrWT), ht_s = smem_addr(sm + kTrHT);
  const uint32_t t_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t id64 = idesc_bf16(128, 64), id16 = idesc_bf16(128, 16);
  const long long plane = n * NRC_W;
  const float inv_n = 1.0f / (float)n;
  float loss_acc = 0.0f;
  uint32_t phase = 0, last = 0;  // last: parity of the latest wait
  bool ok = true;
  // one MMA step of the group: issue (thread 0 of the group), wait, agree
  auto step = [&](auto&& issue) -> bool {
    if (r == 0) issue();
    // warp-uniform, so that the warp-collective TMEM loads run in all lanes or none
    const bool done = __all_sync(0xffffffffu, mbar_wait(bar, last = phase, limit));
    phase ^= 1u;
    tc_fence_after();
    return done;
  };
  const long long n_tiles = (n + 127) / 128;
  for (long long tile = (long long)blockIdx.x * kTrGroups + g; tile < n_tiles && ok;
       tile += (long long)gridDim.x * kTrGroups) {
    const long long row = tile * 128 + r;
    const bool live = row < n;
    // ---- encoding -> X_0
    {
      float rr[NRC_RAW];
#pragma unroll
      for (int k = 0; k < NRC_RAW; ++k) rr[k] = live ? raw[row * NRC_RAW + k] : 0.0f;
      uint32_t w[32];
      nrc_encode_packed(rr, box.lo, box.inv_ext, live, w);
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
        put_chunk(Xt, r, c8, make_uint4(w[4 * c8], w[4 * c8 + 1], w[4 * c8 + 2], w[4 * c8 + 3]),
                  live ? X + row * NRC_W : nullptr);
    }
    fence_async_smem();
    tc_fence_before();
    ok = group_sync_and(g, true);
    // ---- forward: X_{l+1} = relu(X_l W_l^T), then the head
    for (int l = 0; l < NRC_HIDDEN && ok; ++l) {
      const bool done = step([&] { issue_k64(tmem, x_s, w_s + (uint32_t)l * 8192u, id64, bar); });
#pragma unroll
      for (int c16 = 0; c16 < 4 && done; ++c16) {
        float v[16];
        tmem_ld16(t_lane + 16u * c16, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float* p = v + 8 * h;
          const uint4 q = make_uint4(pack_relu_bf16(p[0], p[1]), pack_relu_bf16(p[2], p[3]),
                                     pack_relu_bf16(p[4], p[5]), pack_relu_bf16(p[6], p[7]));
          put_chunk(Xt, r, 2 * c16 + h, q, live ? X + (l + 1) * plane + row * NRC_W : nullptr);
        }
      }
      fence_async_smem();
      tc_fence_before();
      ok = group_sync_and(g, done);
    }
    if (!ok) break;
    {
      const bool done = step([&] { issue_k64(tmem, x_s, h_s, id16, bar); });
      float y[16];
      if (done) tmem_ld16(t_lane, y);
      float dy[3] = {0.f, 0.f, 0.f};
      if (live && done) {
#pragma unroll
        for (int c = 0; c < NRC_OUT; ++c) {
          const float tv = target[row * 3 + c];
          const float den = y[c] * y[c] + 0.01f;
          const float diff = y[c] - tv;
          loss_acc += diff * diff / den * inv_n;
          dy[c] = 2.0f * diff / den * inv_n;
        }
      }
      // head delta: the K = 16 operand tile (columns 0..2) and dZ_5 (64 columns, 3 used)
      const uint4 q0 = make_uint4(pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], 0.f), 0u, 0u);
      *reinterpret_cast<uint4*>(Yt + core16_off(r, 0)) = q0;
      *reinterpret_cast<uint4*>(Yt + core16_off(r, 8)) = make_uint4(0u, 0u, 0u, 0u);
      if (live) {
        uint4* d5 = reinterpret_cast<uint4*>(dZ + NRC_HIDDEN * plane + row * NRC_W);
        d5[0] = q0;
#pragma unroll
        for (int k8 = 1; k8 < 8; ++k8) d5[k8] = make_uint4(0u, 0u, 0u, 0u);
      }
      fence_async_smem();
      tc_fence_before();
      ok = group_sync_and(g, done);
    }
    if (!ok) break;
    // ---- backward: dX_5 = dY Wh, then dZ_l, dX_l for l = 4 .. 0
    {
      const bool done = step([&] { issue_k16(tmem, y_s, ht_s, id64, bar); });
      ok = done;  // agreed below together with the first delta
    }
    for (int l = NRC_HIDDEN - 1; l >= 0; --l) {
      // dZ_l = dX_{l+1} * [X_{l+1} > 0] (X_{l+1} as written by this thread above)
      const uint4* xg = reinterpret_cast<const uint4*>(X + (l + 1) * plane + row * NRC_W);
#pragma unroll
      for (int c16 = 0; c16 < 4 && ok; ++c16) {
        float v[16];
        tmem_ld16(t_lane + 16u * c16, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k8 = 2 * c16 + h;
          const uint4 xq = live ? xg[k8] : make_uint4(0u, 0u, 0u, 0u);
          const uint32_t xw[4] = {xq.x, xq.y, xq.z, xq.w};
          uint32_t dq[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float d0 = bf16_lo(xw[e]) > 0.f ? v[8 * h + 2 * e] : 0.f;
            const float d1 = bf16_hi(xw[e]) > 0.f ? v[8 * h + 2 * e + 1] : 0.f;
            dq[e] = pack_bf16(d0, d1);
          }
          put_chunk(Xt, r, k8, make_uint4(dq[0], dq[1], dq[2], dq[3]),
                    live ? dZ + l * plane + row * NRC_W : nullptr);
        }
      }
      fence_async_smem();
      tc_fence_before();
      ok = group_sync_and(g, ok);
      if (!ok || l == 0) break;
      ok = step([&] { issue_k64(tmem, x_s, wt_s + (uint32_t)l * 8192u, id64, bar); });
    }
    if (!ok) break;
  }
  if (!ok) {
    if (r == 0) atomicCAS(status, 0, PT_ERR_TIMEOUT);
    mbar_wait(bar, last, kWaitLimit);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
  if (lane == 0 && loss_acc != 0.0f) atomicAdd(loss, loss_acc);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*slot), "r"(kTrCols) : "memory");
  }
}

// ---------------------------------------------------------------- training: weight gradients
// dW_l[o][i] += sum_b dZ_l[b][o] X_l[b][i]: split-K over blocks (blockIdx.y = layer,
// the head is layer 5 with o < 3).  The batch is the K dimension: each 64-record
// step loads dZ_l^T (A: o x b, rows 64..127 zero so that M = 128) and X_l^T
// (B: i x b) transposed into K-major tiles and accumulates D (o x i, FP32) in
// TMEM over the block's records; the block then adds D to dW.
constexpr uint32_t kWgA = 0, kWgB = 16384, kWgBar = kWgB + 8192, kWgSlot = kWgBar + 8;
constexpr uint32_t kWgSmem = 40 * 1024;  // > what is used: at most 5 blocks (320 TMEM columns) per SM

__global__ void __launch_bounds__(128) nrc_wgrad_tc_kernel(const __nv_bfloat16* __restrict__ X,
                                                           const __nv_bfloat16* __restrict__ dZ, long long n,
                                                           long long chunk, float* __restrict__ dW,
                                                           int* __restrict__ status, unsigned limit) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* sm = tc_smem_raw + ((1024u - (smem_addr(tc_smem_raw) & 1023u)) & 1023u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kWgBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kWgSlot);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int l = blockIdx.y;
  const long long plane = n * NRC_W;
  const unsigned short* Zl = reinterpret_cast<const unsigned short*>(dZ + l * plane);
  const unsigned short* Xl = reinterpret_cast<const unsigned short*>(X + l * plane);
  const long long b_begin = (long long)blockIdx.x * chunk;
  const long long b_end = b_begin + chunk < n ? b_begin + chunk : n;
  // rows 64..127 of A stay zero
  for (int idx = tid; idx < 16384 / 16; idx += blockDim.x) reinterpret_cast<uint4*>(sm + kWgA)[idx] = make_uint4(0, 0, 0, 0);
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(64u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t a_s = smem_addr(sm + kWgA), b_s = smem_addr(sm + kWgB);
  uint32_t phase = 0, last = 0;  // last: parity of the latest wait
  bool ok = true, any = false;
  for (long long b0 = b_begin; b0 < b_end && ok; b0 += 64) {
    // record rb = tid / 2 of the step, half h = tid % 2 of its 64 columns
    const int rb = tid >> 1, h = tid & 1;
    const long long b = b0 + rb;
    uint4 zq[4], xq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      zq[q] = b < b_end ? reinterpret_cast<const uint4*>(Zl + b * NRC_W + 32 * h)[q] : make_uint4(0, 0, 0, 0);
      xq[q] = b < b_end ? reinterpret_cast<const uint4*>(Xl + b * NRC_W + 32 * h)[q] : make_uint4(0, 0, 0, 0);
    }
    const unsigned short* zs = reinterpret_cast<const unsigned short*>(zq);
    const unsigned short* xs = reinterpret_cast<const unsigned short*>(xq);
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int c = 32 * h + e;  // o for A, i for B
      *reinterpret_cast<unsigned short*>(sm + kWgA + core_off(c, rb)) = zs[e];
      *reinterpret_cast<unsigned short*>(sm + kWgB + core_off(c, rb)) = xs[e];
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
        umma_bf16(tmem, umma_desc(a_s + 256u * s2, kLBO, kSBO), umma_desc(b_s + 256u * s2, kLBO, kSBO),
                  idesc_bf16(128, 64), (any || s2 > 0) ? 1u : 0u);
      umma_commit(bar);
    }
    any = true;
    const bool done = mbar_wait(bar, last = phase, limit);
    phase ^= 1u;
    tc_fence_after();
    tc_fence_before();
    ok = __syncthreads_and(done) != 0;  // the tiles may be overwritten after this
  }
  if (!ok) {
    if (tid == 0) atomicCAS(status, 0, PT_ERR_TIMEOUT);
    mbar_wait(bar, last, kWaitLimit);
  } else if (any && warp < 2) {
    // rows o = 32 warp + lane of D (lanes 0..63): add to dW_l
    float* dWl = dW + (size_t)l * NRC_W * NRC_W;
    const int o = 32 * warp + (tid & 31);
    const int o_lim = l < NRC_HIDDEN ? NRC_W : NRC_OUT;
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16u * c16, v);
      if (o < o_lim) {
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(&dWl[o * NRC_W + 16 * c16 + e], v[e]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u) : "memory");
  }
}

}  // namespace

int cache_infer_tc(const float* raw, float* rgb, long long n, const NrcBox& box, const __nv_bfloat16* Wb, int* status,
                   unsigned wait_limit, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    if (cudaFuncSetAttribute(nrc_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) !=
        cudaSuccess)
      return PT_ERR_CUDA;
    attr = 1;
  }
  const long long tiles = (n + 127) / 128;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (tiles + kGroups - 1) / kGroups;  // one CTA per SM at most (all of its TMEM)
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  nrc_infer_tc_kernel<<<(unsigned)grid, 128 * kGroups, kTcSmem, st>>>(raw, n, box, Wb, rgb, status,
                                                                      wait_limit);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}

}  // namespace ptgb

namespace ptgb {
int cache_train_fb_tc(const float* raw, const float* target, long long n, const NrcBox& box, const __nv_bfloat16* Wb,
                      __nv_bfloat16* X, __nv_bfloat16* dZ, float* loss, int* status, unsigned wait_limit,
                      cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    if (cudaFuncSetAttribute(nrc_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrSmem) !=
        cudaSuccess)
      return PT_ERR_CUDA;
    attr = 1;
  }
  const long long tiles = (n + 127) / 128;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (tiles + kTrGroups - 1) / kTrGroups;
  if (grid > sms) grid = sms;
  if (grid < 1) grid = 1;
  nrc_train_tc_kernel<<<(unsigned)grid, 128 * kTrGroups, kTrSmem, st>>>(raw, target, n, box, Wb, X, dZ, loss, status,
                                                                        wait_limit);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
}  // namespace ptgb

namespace ptgb {
int cache_wgrad_tc(const __nv_bfloat16* X, const __nv_bfloat16* dZ, long long n, long long chunk, float* dW,
                   int* status, unsigned wait_limit, cudaStream_t st) {
  static int attr = 0;
  if (!attr) {
    if (cudaFuncSetAttribute(nrc_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem) !=
        cudaSuccess)
      return PT_ERR_CUDA;
    attr = 1;
  }
  const dim3 grid((unsigned)((n + chunk - 1) / chunk), NRC_HIDDEN + 1);
  nrc_wgrad_tc_kernel<<<grid, 128, kWgSmem, st>>>(X, dZ, n, chunk, dW, status, wait_limit);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
}  // namespace ptgb
