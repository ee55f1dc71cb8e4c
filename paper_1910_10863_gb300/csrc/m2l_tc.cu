// Tensor-core M2L for the mixed-precision matvec (tcgen05, sm_103a).
//
// The M2L translation of Sec. 3.2 depends only on the offset between target and
// source box, so at one level the translations form one small dense operator
// T_o per offset o (40 of them), shared by every box pair at that offset.
// Complex numbers are embedded as real 2P-vectors [Re; Im] and
// T_o as the real 2P x 2P matrix [[Re T, -Im T], [Im T, Re T]].
//
// One CTA owns a tile of 128 target boxes (the MMA's M dimension).  For every
// offset present in the tile it gathers the source multipole of each target
// (times the image phase alpha^m) as row t of the A operand, while B holds T_o
// (row = output coefficient, K-major).  Both operands are split into three
// BF16 parts x = x0 + x1 + x2 and the six products of order <= 2
// (A0B0, A0B1, A1B0, A0B2, A1B1, A2B0) accumulate in FP32 in tensor memory
// across all offsets, which keeps FP32-level accuracy.  The epilogue adds the
// tile's local expansions into L (which already holds the L2L contribution).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int TILE = 128;

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

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  r -= __bfloat162float(b);
  c = __float2bfloat16_rn(r);
}

template <int KP>
__global__ void __launch_bounds__(TILE) m2l_tc_kernel(int P, const int* __restrict__ tile_box,
                                                      const int* __restrict__ tile_noff,
                                                      const int* __restrict__ tile_offs,
                                                      const int* __restrict__ tile_src,
                                                      const int* __restrict__ tile_img,
                                                      const __nv_bfloat16* __restrict__ Bsplit,
                                                      const cplxf* __restrict__ M, cplx alpha, cplxf* __restrict__ L,
                                                      int* __restrict__ err) {
  constexpr int NCOL = KP <= 32 ? 32 : (KP <= 64 ? 64 : 128);   // TMEM columns (power of two)
  constexpr uint32_t SBO = (KP / 8) * 128;
  constexpr uint32_t IDESC = idesc_bf16(TILE, KP);
  extern __shared__ __align__(1024) unsigned char smraw[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smraw);          // 3 x TILE x KP
  __nv_bfloat16* sB = sA + 3 * TILE * KP;                                // 3 x KP x KP
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 3 * KP * KP);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;

  const int tile = blockIdx.x;
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int noff = tile_noff[tile];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // zero the A tiles once (padding columns stay zero)
  {
    uint4* p = reinterpret_cast<uint4*>(sA);
    const int n16 = 3 * TILE * KP * 2 / 16;
    for (int i = t; i < n16; i += TILE) p[i] = make_uint4(0, 0, 0, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int tgt = tile_box[tile * TILE + t];
  uint32_t phase = 0;
  bool ok = true;

  for (int oi = 0; oi < noff && ok; ++oi) {
    const int o = tile_offs[tile * 49 + oi];
    const size_t ti = ((size_t)tile * 49 + oi) * TILE + t;
    const int src = tile_src[ti];
    // A row t: alpha^m M(src) as [Re; Im], three BF16 parts
    if (src >= 0) {
      const int m = tile_img[ti];
      cplxf ph{1.f, 0.f};
      if (m == 1) ph = to_f(alpha);
      else if (m == -1) ph = to_f(cdiv(cplx{1, 0}, alpha));
      for (int n = 0; n < P; ++n) {
        const cplxf v = ph * M[(size_t)src * P + n];
        __nv_bfloat16 a0, a1, a2;
        split3(v.re, a0, a1, a2);
        const uint32_t oR = canon(t, n, KP) >> 1;
        sA[oR] = a0;
        sA[TILE * KP + oR] = a1;
        sA[2 * TILE * KP + oR] = a2;
        split3(v.im, a0, a1, a2);
        const uint32_t oI = canon(t, P + n, KP) >> 1;
        sA[oI] = a0;
        sA[TILE * KP + oI] = a1;
        sA[2 * TILE * KP + oI] = a2;
      }
    } else {
      for (int n = 0; n < 2 * P; ++n) {
        const uint32_t off = canon(t, n, KP) >> 1;
        const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
        sA[off] = z;
        sA[TILE * KP + off] = z;
        sA[2 * TILE * KP + off] = z;
      }
    }
    // B = T_o, three BF16 parts already in the canonical layout
    {
      const uint4* g = reinterpret_cast<const uint4*>(Bsplit + (size_t)o * 3 * KP * KP);
      uint4* s = reinterpret_cast<uint4*>(sB);
      const int n16 = 3 * KP * KP * 2 / 16;
      for (int i = t; i < n16; i += TILE) s[i] = g[i];
    }
    // make the generic-proxy shared-memory writes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      for (int q = 0; q < 6; ++q) {
        const uint32_t abase = smem_u32(sA + pa[q] * TILE * KP);
        const uint32_t bbase = smem_u32(sB + pb[q] * KP * KP);
        for (int kk = 0; kk < KP / 16; ++kk) {
          const uint64_t ad = sdesc(abase + kk * 256, 128, SBO);
          const uint64_t bd = sdesc(bbase + kk * 256, 128, SBO);
          const uint32_t acc = (oi > 0 || q > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
    }
    // bounded wait for the MMAs of this offset (their smem operands are reused next)
    {
      uint32_t done = 0;
      long spins = 0;
      while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
        if (!done && ++spins > (1L << 24)) {
          s_fail = 1;
          break;
        }
      }
      phase ^= 1u;
    }
    __syncthreads();
    ok = (s_fail == 0);            // uniform across the CTA
  }
  if (!ok && t == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && noff > 0) {            // CTA-uniform: every warp runs the collective loads
    float* Lr = reinterpret_cast<float*>(L);
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < KP; c0 += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                     "=r"(v[7])
                   : "r"(lane_addr + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (tgt >= 0) {
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + j;
          if (c < P) Lr[2 * ((size_t)tgt * P + c)] += __uint_as_float(v[j]);
          else if (c < 2 * P) Lr[2 * ((size_t)tgt * P + (c - P)) + 1] += __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
  }
}

uint16_t bf16_bits(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t*>(&b);
}
float bf16_float(uint16_t u) {
  uint32_t w = (uint32_t)u << 16;
  float f;
  std::memcpy(&f, &w, 4);
  return f;
}

}  // namespace

int tc_kpad(int P) { return ((2 * P + 15) / 16) * 16; }

// Host: operator tiles of one level in the canonical layout, three BF16 parts
// split from the FP64 table T [49][P][P] (row = target coefficient).
std::vector<uint16_t> tc_build_operator(const std::vector<cplx>& T, int P) {
  const int kp = tc_kpad(P);
  std::vector<uint16_t> out((size_t)49 * 3 * kp * kp, 0);
  for (int o = 0; o < 49; ++o) {
    for (int c = 0; c < 2 * P; ++c)
      for (int k = 0; k < 2 * P; ++k) {
        const cplx v = T[((size_t)o * P + (c % P)) * P + (k % P)];
        double x;
        if (c < P && k < P) x = v.re;
        else if (c < P) x = -v.im;
        else if (k < P) x = v.im;
        else x = v.re;
        const float x0f = (float)x;
        const uint16_t b0 = bf16_bits(x0f);
        const double r1 = x - (double)bf16_float(b0);
        const uint16_t b1 = bf16_bits((float)r1);
        const double r2 = r1 - (double)bf16_float(b1);
        const uint16_t b2 = bf16_bits((float)r2);
        const size_t base = (size_t)o * 3 * kp * kp;
        const uint32_t off = canon(c, k, kp) >> 1;
        out[base + off] = b0;
        out[base + (size_t)kp * kp + off] = b1;
        out[base + 2 * (size_t)kp * kp + off] = b2;
      }
  }
  return out;
}

cudaError_t k_m2l_tc(pfmbem* h, int l, const cplxf* M, cplxf* L) {
  Level& a = h->lev[l];
  if (a.tc_ntile == 0) return cudaSuccess;
  const int kp = tc_kpad(a.P);
  const size_t smem = (size_t)3 * TILE * kp * 2 + (size_t)3 * kp * kp * 2 + 16;
  cudaStream_t st = h->stream;
#define PF_TC_CASE(KP)                                                                                    \
  case KP:                                                                                                \
    cudaFuncSetAttribute(m2l_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    m2l_tc_kernel<KP><<<a.tc_ntile, TILE, smem, st>>>(a.P, a.tc_box, a.tc_noff, a.tc_offs, a.tc_src,     \
                                                      a.tc_img, reinterpret_cast<const __nv_bfloat16*>(a.tc_B),  \
                                                      M, h->alpha, L, h->tc_err);                         \
    break;
  switch (kp) {
    PF_TC_CASE(32)
    PF_TC_CASE(48)
    PF_TC_CASE(64)
    PF_TC_CASE(80)
    PF_TC_CASE(96)
    PF_TC_CASE(112)
    PF_TC_CASE(128)
    default:
      return cudaErrorInvalidValue;
  }
#undef PF_TC_CASE
  return cudaGetLastError();
}
