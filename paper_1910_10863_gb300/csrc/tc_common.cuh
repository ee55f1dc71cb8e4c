// tcgen05 helpers shared by the tensor-core M2L kernels (sm_103a): operand
// layout in shared memory, descriptors and the three-way BF16 split.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tc {

constexpr int TILE = 128;   // target boxes per tile = the MMA's M dimension

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) in a K-major operand tile without swizzle:
// 8-row x 16-byte core matrices, consecutive along K (LBO = 128 B), 8-row
// groups SBO = (kp / 8) * 128 B apart.
__host__ __device__ __forceinline__ uint32_t canon(int r, int k, int kp) {
  return (uint32_t)((((r >> 3) * (kp >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, version 1 in
// bits 46-47, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// x = a + b + c in BF16 parts (each the rounding of what the previous left).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  r -= __bfloat162float(b);
  c = __float2bfloat16_rn(r);
}

// K padded to the MMA's K step of 16 for 2P real components.
__host__ __device__ constexpr int kpad(int P) { return ((2 * P + 15) / 16) * 16; }

// First accumulator column of the imaginary parts in the single-launch
// product's layout: P rounded up to 8 (for odd P, imrow(P) + P <= kpad(P)).
__host__ __device__ constexpr int imrow(int P) { return ((P + 7) / 8) * 8; }

}  // namespace tc
