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
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

#include "tc_common.cuh"

namespace {

using tc::TILE;
using tc::canon;
using tc::idesc_bf16;
using tc::sdesc;
using tc::smem_u32;
using tc::split3;

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

  // blockIdx.x = tile, blockIdx.y = group of offsets handled by this CTA
  const int tile = blockIdx.x;
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int ntot = tile_noff[tile];
  const int og = (ntot + gridDim.y - 1) / gridDim.y;
  const int ofirst = blockIdx.y * og;
  const int noff = max(0, min(ntot, ofirst + og) - ofirst);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int tgt = tile_box[tile * TILE + t];
  uint32_t phase = 0;
  bool ok = true;

  for (int oj = 0; oj < noff && ok; ++oj) {
    const int oi = ofirst + oj;
    const int o = tile_offs[tile * 49 + oi];
    const size_t ti = ((size_t)tile * 49 + oi) * TILE + t;
    const int src = tile_src[ti];
    // A row t: alpha^m M(src) as [Re; Im] (zero row without a source), three
    // BF16 parts; one 16-byte store per core-matrix row (8 consecutive k)
    {
      const int m = src >= 0 ? tile_img[ti] : 0;
      cplxf ph{1.f, 0.f};
      if (m == 1) ph = to_f(alpha);
      else if (m == -1) ph = to_f(cdiv(cplx{1, 0}, alpha));
      const cplxf* Ms = M + (size_t)(src >= 0 ? src : 0) * P;
      for (int g = 0; g < KP / 8; ++g) {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          float x[2];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int k = 8 * g + 2 * jj + hh;
            float v = 0.f;
            if (src >= 0 && k < 2 * P) {
              const cplxf z = ph * Ms[k < P ? k : k - P];
              v = k < P ? z.re : z.im;
            }
            x[hh] = v;
          }
          __nv_bfloat16 a0, a1, a2, b0, b1, b2;
          split3(x[0], a0, a1, a2);
          split3(x[1], b0, b1, b2);
          w0[jj] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(b0) << 16);
          w1[jj] = (uint32_t)__bfloat16_as_ushort(a1) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
          w2[jj] = (uint32_t)__bfloat16_as_ushort(a2) | ((uint32_t)__bfloat16_as_ushort(b2) << 16);
        }
        const uint32_t off = canon(t, 8 * g, KP) >> 4;    // in 16-byte units
        reinterpret_cast<uint4*>(sA)[off] = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        reinterpret_cast<uint4*>(sA + TILE * KP)[off] = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        reinterpret_cast<uint4*>(sA + 2 * TILE * KP)[off] = make_uint4(w2[0], w2[1], w2[2], w2[3]);
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
          const uint32_t acc = (oj > 0 || q > 0 || kk > 0) ? 1u : 0u;
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
      if (tgt >= 0) {   // several CTAs (offset groups) add into the same target
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + j;
          if (c < P) atomicAdd(&Lr[2 * ((size_t)tgt * P + c)], __uint_as_float(v[j]));
          else if (c < 2 * P) atomicAdd(&Lr[2 * ((size_t)tgt * P + (c - P)) + 1], __uint_as_float(v[j]));
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

// x = b0 + b1 + b2 in BF16 parts, split in FP64.
__device__ __forceinline__ void split3d(double x, __nv_bfloat16& b0, __nv_bfloat16& b1, __nv_bfloat16& b2) {
  b0 = __float2bfloat16_rn((float)x);
  const double r1 = x - (double)__bfloat162float(b0);
  b1 = __float2bfloat16_rn((float)r1);
  const double r2 = r1 - (double)__bfloat162float(b1);
  b2 = __float2bfloat16_rn((float)r2);
}

// The operators of the single-launch FP32 product, for its interleaved layout:
// K index 2c + 0 / 2c + 1 multiplies the real / imaginary part of source
// coefficient c; output row n < Pu gives the real part of target coefficient
// n and row imrow + n its imaginary part:
//   row n:         [Re T_nc, -Im T_nc],   row imrow + n: [Im T_nc, Re T_nc].
// Used block of Pu coefficients from offset O of the FP64 table T [49][S][S].
// One thread per (offset, output, source coefficient).
__global__ void tc_split_fused_kernel(int Pu, int S, int O, int kp, int imrow, const cplx* __restrict__ T,
                                      __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)Pu * Pu;
  if (i >= 49 * n2) return;
  const int o = (int)(i / n2), rem = (int)(i % n2), n = rem / Pu, c = rem % Pu;
  const cplx v = T[((size_t)o * S + O + n) * S + O + c];
  const size_t base = (size_t)o * 3 * kp * kp;
  const double val[4] = {v.re, -v.im, v.im, v.re};
  const int rows[2] = {n, imrow + n};
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat16 b[3];
    split3d(val[q], b[0], b[1], b[2]);
    const uint32_t off = canon(rows[q >> 1], 2 * c + (q & 1), kp) >> 1;
    for (int j = 0; j < 3; ++j) out[base + (size_t)j * kp * kp + off] = b[j];
  }
}

// Operator tiles of one level in the canonical layout: three BF16 parts split
// (in FP64) from the FP64 table T [49][S][S] (row = target coefficient) of the
// real-embedded complex operator, its used block of Pu coefficients from
// offset O.  One thread per (offset, row, column).
__global__ void tc_split_kernel(int Pu, int S, int O, int kp, const cplx* __restrict__ T,
                                __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)(2 * Pu) * (2 * Pu);
  if (i >= 49 * n2) return;
  const int o = (int)(i / n2), rem = (int)(i % n2), c = rem / (2 * Pu), k = rem % (2 * Pu);
  const cplx v = T[((size_t)o * S + O + (c % Pu)) * S + O + (k % Pu)];
  double x;
  if (c < Pu && k < Pu) x = v.re;
  else if (c < Pu) x = -v.im;
  else if (k < Pu) x = v.im;
  else x = v.re;
  const __nv_bfloat16 b0 = __float2bfloat16_rn((float)x);
  const double r1 = x - (double)__bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn((float)r1);
  const double r2 = r1 - (double)__bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn((float)r2);
  const size_t base = (size_t)o * 3 * kp * kp;
  const uint32_t off = canon(c, k, kp) >> 1;
  out[base + off] = b0;
  out[base + (size_t)kp * kp + off] = b1;
  out[base + 2 * (size_t)kp * kp + off] = b2;
}

}  // namespace

int tc_kpad(int P) { return tc::kpad(P); }

cudaError_t k_tc_build_operator(pfmbem* h, int l) {
  Level& a = h->lev[l];
  const int kp = tc_kpad(a.P);
  cudaError_t e = cudaMemsetAsync(a.tc_B, 0, sizeof(uint16_t) * 49 * 3 * (size_t)kp * kp, h->stream);
  if (e != cudaSuccess) return e;
  const int64_t n = 49LL * (2 * a.P) * (2 * a.P);
  prof_begin(h, PH_SETUP);
  tc_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(a.P, a.P, 0, kp, a.m2l,
                                                                      reinterpret_cast<__nv_bfloat16*>(a.tc_B));
  prof_end(h, PH_SETUP);
  return cudaGetLastError();
}

// The central Pu-coefficient block for the single-launch FP32 product, in its
// interleaved layout.
cudaError_t k_tc_build_operator_fused(pfmbem* h, int l, int Pu) {
  Level& a = h->lev[l];
  const int kp = tc_kpad(Pu);
  cudaError_t e = cudaMemsetAsync(a.tc_Bf, 0, sizeof(uint16_t) * 49 * 3 * (size_t)kp * kp, h->stream);
  if (e != cudaSuccess) return e;
  const int64_t n = 49LL * Pu * Pu;
  prof_begin(h, PH_SETUP);
  tc_split_fused_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      Pu, a.P, (a.P - Pu) / 2, kp, tc::imrow(Pu), a.m2l, reinterpret_cast<__nv_bfloat16*>(a.tc_Bf));
  prof_end(h, PH_SETUP);
  return cudaGetLastError();
}

cudaError_t k_m2l_tc(pfmbem* h, int l, const cplxf* M, cplxf* L) {
  Level& a = h->lev[l];
  if (a.tc_ntile == 0) return cudaSuccess;
  const int kp = tc_kpad(a.P);
  const size_t smem = (size_t)3 * TILE * kp * 2 + (size_t)3 * kp * kp * 2 + 16;
  cudaStream_t st = h->stream;
  // split every tile's offsets over enough CTAs to cover the GPU about twice
  int sms = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int groups = std::max(1, std::min(4, (2 * sms + a.tc_ntile - 1) / a.tc_ntile));
  const dim3 grid(a.tc_ntile, groups);
#define PF_TC_CASE(KP)                                                                                    \
  case KP:                                                                                                \
    cudaFuncSetAttribute(m2l_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    m2l_tc_kernel<KP><<<grid, TILE, smem, st>>>(a.P, a.tc_box, a.tc_noff, a.tc_offs, a.tc_src,           \
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
