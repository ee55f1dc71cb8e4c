// The cached matrix-vector product (I - A) x of eq. 9 as ONE cooperative launch.
//
// The per-stage path launches some twenty small kernels per product (gather,
// P2M, one M2M per level, L2L and M2L per level, L2P, near field, fiber
// blocks); at the sizes of a fundamental block most of them are latency-bound.
// Here one grid of co-resident blocks runs the stages back to back and
// separates them with a device-wide barrier:
//
//   A   gather the densities into tree order (alpha^{-m0} phase), P2M and
//       clear the local expansions of levels 1..D (warp per leaf); at the
//       same time a share of the blocks applies the same-fiber blocks of
//       eq. 9 to x and writes them to y: a regular-polygon fiber whose
//       element count is a power of two by FFT (block per fiber), the others
//       by cached rows (block per chunk of 32 rows)
//   B_l M2M into level l = D-1 .. 0 (warp per box, or per output coefficient
//       where the boxes are few); the root stage forms L(0) directly from the
//       four level-1 multipoles through the folded operator R T_0.  The
//       cached near-field sums of all elements are spread evenly over these
//       stages, whose few boxes leave most warps idle        (warp per element)
//   D_l L2L from the parent (warp per box or per coefficient) and M2L (warp
//       per pair, or block per chunk of pairs with one translation offset and
//       T_o staged in shared memory), both added atomically into L(l)
//   E   L2P plus the near-field sums, and the combination of eq. 9 added to
//       the fiber part already in y                           (warp per element)
//
// Warp-level items are dealt round-robin over the blocks (item i to block
// i mod grid), so that a stage with few items still spreads over all SMs: on
// GB300 the FP64 pipe of one SM sub-partition executes a warp-wide DFMA only
// every few dozen cycles, and a stage is as slow as its busiest SM.
//
// The barrier is a counter plus a generation word in device memory.  The
// cooperative launch guarantees that every block is resident, so every wait
// ends; each wait is nevertheless bounded (one second of %globaltimer), after which the
// block records an error flag and returns, and the host reports
// PFMBEM_ETIMEOUT instead of a result.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace {

constexpr int FB = 256;          // threads per block
constexpr int FW = FB / 32;      // warps per block

// Device time in nanoseconds.
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Threads and warps of the running block: the single-launch product runs with
// 256 threads per block, or 512 in its tensor-core form (one block per SM)
__device__ __forceinline__ int nt() { return (int)blockDim.x; }
__device__ __forceinline__ int nw() { return (int)(blockDim.x >> 5); }
constexpr int TSP = 49;          // largest order count P whose M2L operator is staged in shared memory
constexpr int TSIZE = TSP * (TSP + 1);

template <class C>
struct FusedArgs {
  int E, D;
  int nroot;                     // root squares in a row along x (level 0 has nroot boxes)
  const int* perm;               // sorted -> original element
  const cplx* ph;                // alpha^{-m0} of every sorted element
  const int* opos;               // original -> sorted
  const cplx* x;                 // input, original order, FP64
  cplx* y;                       // output, original order, FP64
  C* dens;                       // sorted (phi', varphi')
  C* Un;                         // sorted near-field part of (U', dU')
  const int* s_li;               // sorted element -> index of its leaf among the non-empty leaves
  int nne[PF_MAXLEVEL + 1];
  int nbox[PF_MAXLEVEL + 1];
  // expansions of level l: P[l] coefficients used, stored in rows of S[l] from
  // offset O[l] on (the FP32 product may run at a lower order than its tables:
  // it then uses their central S-by-S sub-blocks; P = S and O = 0 otherwise)
  int P[PF_MAXLEVEL + 1];
  int S[PF_MAXLEVEL + 1];
  int O[PF_MAXLEVEL + 1];
  int nch[PF_MAXLEVEL + 1];      // M2L chunks (pairs of one offset) per level
  const int* ne[PF_MAXLEVEL + 1];
  const int* bb[PF_MAXLEVEL + 1];
  const int* be[PF_MAXLEVEL + 1];
  const int* ch_off[PF_MAXLEVEL + 1];
  const int* ch_beg[PF_MAXLEVEL + 1];
  const int* ch_end[PF_MAXLEVEL + 1];
  const int* pr_tgt[PF_MAXLEVEL + 1];
  const int* pr_src[PF_MAXLEVEL + 1];
  const int* pr_img[PF_MAXLEVEL + 1];
  const int* pr_off[PF_MAXLEVEL + 1];    // translation offset per pair
  int npair[PF_MAXLEVEL + 1];
  const C* m2m[PF_MAXLEVEL + 1];     // at the parent level: [q][m child][n parent]
  const C* l2l[PF_MAXLEVEL + 1];     // at the parent level: [q][m parent][n child]
  const C* m2lt[PF_MAXLEVEL + 1];    // [o][n source][l target]
  C* M[PF_MAXLEVEL + 1];
  C* L[PF_MAXLEVEL + 1];
  const C* root;                     // [l][n], lattice-sum translation at the root
  const C* rootc;                    // [u < 4 P_1][l < P_0], R T_0: L(0) from the level-1 multipoles
  int top3;                          // 1: the level-2 stage also forms M(1), and L(0) is never formed
  const C* m2m31;                    // [n < P_1][u < 16 P_3], T_1 T_2
  const C* root1;                    // [q][n < P_1][u < 4 P_1], L2L_q R T_0: L(1) from the level-1 multipoles
  const C* p2m;                      // [E][2][P_D]
  const C* l2p;                      // [2][P_D][E], coefficient-major
  const int64_t* nc_base;
  const int* nc_sbase;
  const longlong2* nr_meta;          // per sorted element: block offset of its near row, (first source << 32) | sources
  // FP32 product: the near rows cut into pieces of at most NR_PIECE sources,
  // each one 16-byte descriptor (offset of its first block, low and high word;
  // its first source in nc_src; (sources << 24) | sorted element), summed
  // atomically into Un (zeroed in stage A); 0 pieces: whole rows
  const int4* nr_piece;
  int npiece;
  const int* nc_src;
  const C* nc_val;
  int nchunk;                        // direct-row chunks (fibers not applied by FFT)
  const int* fb_chunk;
  int nfft;                          // fibers applied by FFT
  const int* fft_fib;
  const int64_t* fh_base;            // [M] first frequency of the fiber's block symbol
  const C* fh_val;                   // [sum N][4] block symbol B^(r,s)(k)
  const C* tw;                       // [512] e^{2 pi i j / 1024}
  const int* foff;
  const int64_t* fb_base;
  const C* fb_val;
  const int* circ;
  cplx alpha, c2;
  int fblk;                          // blocks applying the same-fiber blocks during stage A (0: all, after P2M)
  int m2l_warp;                      // M2L one warp per pair (1) or one block per staged chunk (0)
  int near_first;                    // measurement: every near-field row in the first B stage
  unsigned long long* bar;           // arrival counter of the device-wide barriers
  int* err;
  unsigned long long wait_ns;        // bound of every barrier wait
  unsigned long long* stamp;         // optional stage end times (ns), written by block 0
  unsigned long long* arrive;        // optional [barrier][block] arrival times (ns)
  unsigned long long* bdone;         // optional [barrier][block] end of the block items (ns)
  const int* done;                   // optional: the product is skipped when *done != 0
  int tws_off;                       // shared-memory offset (in C) of the twiddle copy of the fiber part
  int treg;                          // shared-memory region (in C) of the staged operators, >= TSIZE
  int tregL;                         // a second region for the L2L operators (0: L2L stages into the first)
  // FP32 product, M2L on the tensor cores (tcgen05) at the levels with tc_kp > 0:
  // tiles of 128 target boxes; block item (tile, group of the tile's offsets)
  int tc_any;
  int tc_kp[PF_MAXLEVEL + 1];            // MMA N = K: 2P padded to 16 (0: CUDA cores)
  int tc_ngrp[PF_MAXLEVEL + 1];          // offset groups per tile
  int tc_ntile[PF_MAXLEVEL + 1];
  const int* tc_box[PF_MAXLEVEL + 1];    // [tile][128] target box, -1 padding
  const int* tc_noff[PF_MAXLEVEL + 1];   // [tile] offsets present
  const int* tc_offs[PF_MAXLEVEL + 1];   // [tile][49] offset ids
  const int* tc_src[PF_MAXLEVEL + 1];    // [tile][49][128] source box, -1: none
  const int* tc_img[PF_MAXLEVEL + 1];    // [tile][49][128] image m of the source
  const uint16_t* tc_B[PF_MAXLEVEL + 1]; // [49][3][kp][kp] BF16 parts of the operators (canonical layout)
  // FP64 product only: the near-field sums in double-float arithmetic (FP32
  // hi + lo pairs), on the FP32 pipes, from these lo parts
  const cplxf* nc_lo;                // lo parts of the near blocks (hi parts: the FP32 copy)
  cplxf* dens_dd;                    // [2][2E] hi and lo parts of the sorted densities
  const cplxf* nc_hi;
  const cplxf* m2lth[PF_MAXLEVEL + 1];   // FP64 product, double-float M2L: hi and lo parts of m2lt
  const cplxf* m2ltl[PF_MAXLEVEL + 1];
  const cplxf* m2mh[PF_MAXLEVEL + 1];    // FP64 product, double-float M2M: hi and lo parts of m2m
  const cplxf* m2ml[PF_MAXLEVEL + 1];
  const cplxf* p2mh;                     // FP64 product, double-float P2M: hi and lo parts of p2m
  const cplxf* p2ml;
  const cplxf* l2lh[PF_MAXLEVEL + 1];    // FP64 product, double-float L2L: hi and lo parts of l2l
  const cplxf* l2ll[PF_MAXLEVEL + 1];
  const cplxf* l2ph;                     // FP64 product, double-float L2P: hi and lo parts of l2p
  const cplxf* l2pl;
  int l2p_dd;                            // measurement (PFMBEM_L2P_DD=1): it measured slower than FP64
  // FP32 product: near-field sums in differences (dlo: lo parts of the sorted
  // densities, rsum: FP64 row sums of the near blocks) and the same-fiber FFTs
  // in FP64 (fh64, tw64: the FP64 block symbols and twiddles)
  cplxf* dlo;
  const cplx* rsum;
  const cplx* fh64;
  const cplx* tw64;
  // FP32 product: row sums of the same-fiber rows applied by rows, split by the
  // parity of the column ([2E rows][2], FP64), for their sums in differences
  const cplx* frs;
};

__device__ __forceinline__ void stage_stamp(unsigned long long* stamp, int k, int bid) {
  if (stamp && bid == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    stamp[k] = t;
  }
}

// alpha^m for m in {-1, 0, 1}; |alpha| = 1, so alpha^{-1} = conj(alpha)
__device__ __forceinline__ cplx phase_m(cplx alpha, int m) {
  return m == 0 ? cplx{1, 0} : (m > 0 ? alpha : conj(alpha));
}

// Loads of values written by other blocks earlier in the same launch bypass L1
// (ld.global.cg), so that no line cached before the barrier is read stale.
__device__ __forceinline__ cplx ldcg(const cplx* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cplx{v.x, v.y};
}
__device__ __forceinline__ cplxf ldcg(const cplxf* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cplxf{v.x, v.y};
}

__device__ __forceinline__ void atomic_add(cplx* p, cplx v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}
__device__ __forceinline__ void atomic_add(cplxf* p, cplxf v) {
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(v.re, v.im));   // one 8-byte vector atomic
}

template <class C>
__device__ __forceinline__ C wsum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_down_sync(0xffffffffu, v.re, o);
    v.im += __shfl_down_sync(0xffffffffu, v.im, o);
  }
  return v;
}

// Barrier over the nb blocks that share the counter bar (the whole grid, or
// one group of blocks of a persistent launch), with a bounded wait; false when
// any block gave up.  One 64-bit arrival counter that only grows: a block's
// arrival is a release add (it publishes the block's writes), whose old value
// tells the barrier's target, the next multiple of nb; the block then polls the
// counter with acquire loads (taking in everyone else's writes) until it
// reaches the target.  Each completed pass adds a multiple of nb, so the
// counter stays aligned as long as only those nb blocks use it; it is cleared
// after a wait ran out.  Optionally records the arrival time (ns) of block bid.
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool group_barrier(unsigned long long* bar, int* err, unsigned long long limit, int nb, int bid,
                              unsigned long long* arrive = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    if (arrive) arrive[bid] = t0;
    int ok = 1;
    const unsigned long long G = (unsigned long long)nb;
    unsigned long long old;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], 1;" : "=l"(old) : "l"(bar) : "memory");
    const unsigned long long target = (old / G + 1) * G;
    while (ld_acquire64(bar) < target) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
    }
    s_ok = ok && *(volatile int*)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// The barrier over the whole grid.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, int* err, unsigned long long limit = 1000000000ull,
                                             unsigned long long* arrive = nullptr) {
  return group_barrier(bar, err, limit, (int)gridDim.x, (int)blockIdx.x, arrive);
}

// acc += sum_m A[m * P] * w[m], m < K (A already offset to the output column),
// two independent accumulators and unrolled loads.
template <class C>
__device__ __forceinline__ C colmv(const C* __restrict__ A, int P, const C* w, int K) {
  C a0{0, 0}, a1{0, 0};
  int m = 0;
#pragma unroll 4
  for (; m + 1 < K; m += 2) {
    a0 += A[(size_t)m * P] * w[m];
    a1 += A[(size_t)(m + 1) * P] * w[m + 1];
  }
  if (m < K) a0 += A[(size_t)m * P] * w[m];
  return a0 + a1;
}

template <class C>
__device__ __forceinline__ C shfl_c(C v, int src) {
  v.re = __shfl_sync(0xffffffffu, v.re, src);
  v.im = __shfl_sync(0xffffffffu, v.im, src);
  return v;
}

// One warp: y[n] = sum_{u < K} A[u P + n] w[u] for every n < P, handed to
// out(n, y[n]).  Full passes of 32 outputs; the last r = P mod 32 outputs are
// shared by 32 / r lane groups that split the u range, their partial sums
// combined by shuffles (P = 37 then costs 1.17 K steps instead of 2 K).
template <class C, class Out>
__device__ __forceinline__ void warp_colmv(const C* A, int P, const C* w, int K, int lane, Out out) {
  const int full = P & ~31;
  for (int n0 = 0; n0 < full; n0 += 32) out(n0 + lane, colmv(A + n0 + lane, P, w, K));
  const int r = P - full;
  if (r == 0) return;
  const int g = 32 / r, grp = lane / r, nr = lane - grp * r;
  C acc{0, 0};
  if (grp < g) {
    const C* Ar = A + full + nr;
#pragma unroll 4
    for (int u = grp; u < K; u += g) acc += Ar[(size_t)u * P] * w[u];
  }
  C s = acc;
  for (int k = 1; k < g; ++k) {
    const C o = shfl_c(acc, k * r + nr);
    s += o;
  }
  if (lane < r) out(full + lane, s);
}

// One warp, two vectors sharing the operator rows: yA[n] = sum_{m < P} T[n P + m]
// wA[m] and yB likewise, handed to out(n, yA[n], yB[n]); the last P mod 32 rows
// are split over lane groups as in warp_colmv.
template <class C, class Out>
__device__ __forceinline__ void warp_rowmv2(const C* T, int P, const C* wA, const C* wB, int lane, Out out) {
  const int full = P & ~31;
  for (int n0 = 0; n0 < full; n0 += 32) {
    const C* row = T + (size_t)(n0 + lane) * P;
    C rA{0, 0}, rB{0, 0};
#pragma unroll 4
    for (int m = 0; m < P; ++m) {
      const C t = row[m];
      rA += t * wA[m];
      rB += t * wB[m];
    }
    out(n0 + lane, rA, rB);
  }
  const int r = P - full;
  if (r == 0) return;
  const int g = 32 / r, grp = lane / r, nr = lane - grp * r;
  C rA{0, 0}, rB{0, 0};
  if (grp < g) {
    const C* row = T + (size_t)(full + nr) * P;
#pragma unroll 4
    for (int m = grp; m < P; m += g) {
      const C t = row[m];
      rA += t * wA[m];
      rB += t * wB[m];
    }
  }
  C sA = rA, sB = rB;
  for (int k = 1; k < g; ++k) {
    const C oA = shfl_c(rA, k * r + nr), oB = shfl_c(rB, k * r + nr);
    sA += oA;
    sB += oB;
  }
  if (lane < r) out(full + lane, sA, sB);
}

// Block-wide copy of n values from global to shared memory with the loads of a
// thread batched ahead of its stores (eight in flight): the copy then costs
// about one L2 round trip instead of one per element the thread moves.
// dst[idx(t)] = src[t]; idx maps the source index to the staged position.
template <class C, class Idx>
__device__ __forceinline__ void stage_copy(C* dst, const C* __restrict__ src, int n, Idx idx) {
  constexpr int U = 8;
  int t = threadIdx.x;
  for (; t + (U - 1) * nt() < n; t += U * nt()) {
    C v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = src[t + u * nt()];
#pragma unroll
    for (int u = 0; u < U; ++u) dst[idx(t + u * nt())] = v[u];
  }
  for (; t < n; t += nt()) dst[idx(t)] = src[t];
}
struct IdxSame {
  __device__ int operator()(int t) const { return t; }
};
struct IdxTranspose {          // [n][l] -> [l][n], P x P
  int P;
  __device__ int operator()(int t) const { return (t % P) * P + t / P; }
};
// The used block of a table with rows of stride S: compact index t (row t / P,
// column t % P) of the staged copy reads src[(t / P) S + t % P].
struct IdxBlock {
  int P, S;
};

template <class C>
__device__ __forceinline__ void stage_copy(C* dst, const C* __restrict__ src, int n, IdxBlock b) {
  constexpr int U = 8;
  int t = threadIdx.x;
  for (; t + (U - 1) * nt() < n; t += U * nt()) {
    C v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = t + u * nt(), r = w / b.P;
      v[u] = src[(size_t)r * b.S + (w - r * b.P)];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) dst[t + u * nt()] = v[u];
  }
  for (; t < n; t += nt()) {
    const int r = t / b.P;
    dst[t] = src[(size_t)r * b.S + (t - r * b.P)];
  }
}

// The used P x P block of a [P source][P target] operator with rows of stride S,
// staged transposed ([target][source]) with batched loads.
template <class C>
__device__ __forceinline__ void stage_copy_bt(C* dst, const C* __restrict__ src, int P, int S) {
  constexpr int U = 8;
  const int n = P * P;
  int t = threadIdx.x;
  for (; t + (U - 1) * nt() < n; t += U * nt()) {
    C v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = t + u * nt(), r = w / P;
      v[u] = src[(size_t)r * S + (w - r * P)];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = t + u * nt(), r = w / P;
      dst[(w - r * P) * P + r] = v[u];
    }
  }
  for (; t < n; t += nt()) {
    const int r = t / P;
    dst[(t - r * P) * P + r] = src[(size_t)r * S + (t - r * P)];
  }
}

// The four quadrant operators of a translation table, stacked: staged row
// u = q Pn + m (q < 4, m < Pn) holds the used columns O .. O + P of table row
// q Sn + On + m (base = table + On S + O; rows of stride S).  Eight loads in
// flight per thread (measured faster than sixteen, 2.1 against 3.1 us for a
// 4 x 37 x 37 stack over 304 blocks).
template <class C>
__device__ __forceinline__ void stage_copy_quad(C* dst, const C* __restrict__ base, int P, int Pn, int S, int Sn) {
  constexpr int U = 8;
  const int n = 4 * Pn * P;
  int t = threadIdx.x;
  for (; t < n; t += U * nt()) {
    C v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int w = t + k * nt();
      if (w < n) {
        const int u = w / P, q = u / Pn;
        v[k] = base[(size_t)(q * Sn + (u - q * Pn)) * S + (w - u * P)];
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (t + k * nt() < n) dst[t + k * nt()] = v[k];
  }
}

// In-place radix-2 FFTs of nseq sequences of length N = 2^lg (N <= 1024)
// held one after another in shared memory, by the whole block:
//   s_q(k) <- sum_j s_q(j) e^{sign 2 pi i j k / N}.
// Decimation in time: bit-reversed order, then lg butterfly passes whose
// twiddles come from the table of e^{2 pi i j / 1024}.
template <class C>
__device__ void block_fft(C* s, int nseq, int lg, int sign, const C* __restrict__ tw) {
  const int N = 1 << lg, half_n = N >> 1;
  __syncthreads();
  for (int t = threadIdx.x; t < nseq * N; t += blockDim.x) {
    const int q = t >> lg, j = t & (N - 1);
    const int k = (int)(__brev((unsigned)j) >> (32 - lg));
    if (j < k) {
      C* sq = s + (q << lg);
      const C v = sq[j];
      sq[j] = sq[k];
      sq[k] = v;
    }
  }
  __syncthreads();
  for (int st = 1; st <= lg; ++st) {
    const int half = 1 << (st - 1), step = 1024 >> st;
    for (int t = threadIdx.x; t < nseq * half_n; t += blockDim.x) {
      const int q = t / half_n, b = t - q * half_n;
      const int pos = b & (half - 1), i = ((b >> (st - 1)) << st) + pos;
      C w = tw[pos * step];
      if (sign < 0) w.im = -w.im;
      C* sq = s + (q << lg);
      const C u = sq[i], v = sq[i + half] * w;
      sq[i] = u + v;
      sq[i + half] = u - v;
    }
    __syncthreads();
  }
}

// Block symbol of a block-circulant fiber block.  The stored row pair R_r
// (r = 0, 1) of the first element gives the blocks b_d^(r,s) = R_r[2d + s]
// with y_e^(r) = sum_{s,d} b_d^(r,s) x_{(e+d) mod N}^(s); with
// X(k) = sum_f x_f e^{-2 pi i k f / N} this is Y^(r)(k) = sum_s B^(r,s)(k) X^(s)(k),
// B^(r,s)(k) = sum_d b_d^(r,s) e^{+2 pi i k d / N}.  One block per fiber.
__global__ void fiber_symbol_kernel(const int* __restrict__ fib_list, const int* __restrict__ foff,
                                    const int64_t* __restrict__ fb_base, const cplx* __restrict__ rows,
                                    const int64_t* __restrict__ fh_base, const cplx* __restrict__ tw,
                                    cplx* __restrict__ fh, cplxf* __restrict__ fhf) {
  extern __shared__ __align__(128) unsigned char smraw[];
  cplx* s = reinterpret_cast<cplx*>(smraw);      // [2][N]
  const int fb = fib_list[blockIdx.x];
  const int N = foff[fb + 1] - foff[fb], lg = __ffs(N) - 1;
  const cplx* R = rows + fb_base[fb];
  cplx* out = fh + 4 * fh_base[fb];
  cplxf* outf = fhf + 4 * fh_base[fb];
  for (int r = 0; r < 2; ++r) {
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int q = t / N, d = t - q * N;
      s[t] = R[(size_t)r * 2 * N + 2 * d + q];
    }
    block_fft(s, 2, lg, +1, tw);
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      const int q = t / N, k = t - q * N;
      out[4 * k + 2 * r + q] = s[t];
      outf[4 * k + 2 * r + q] = to_f(s[t]);
    }
  }
}

// L(0) from the four level-1 multipoles: Rc = R T_0, with R the periodic root
// translation and T_0 the level-1 -> root M2M, stored [u][l] for the 4 P_1
// child coefficients u, so that the fused product never forms M(0).  One
// warp per entry (lanes over the P_0 terms), FP64, with an FP32 copy.
// With nr roots in a row, R is the operator between all roots ([nr P0][nr P0]) and
// row u = (level-1 box ch, coefficient m) of the fold, ch = 4 j + q below root j,
// meets column t = (root i, coefficient a): rc[u][t] = sum_n R[t][j P0 + n] T_0^q[m][n].
__global__ void root_fold_kernel(int P0, int K, int nr, const cplx* __restrict__ R, const cplx* __restrict__ m2m0,
                                 cplx* __restrict__ rc, cplxf* __restrict__ rcf) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int NP = nr * P0, P1 = K / 4;
  if (i >= NP * nr * K) return;
  const int u = i / NP, t = i - u * NP;
  const int ch = u / P1, m = u - ch * P1, j = ch >> 2, q = ch & 3;
  const cplx* Rr = R + (size_t)t * NP + (size_t)j * P0;
  const cplx* Tq = m2m0 + (size_t)(q * P1 + m) * P0;
  cplx s{0, 0};
  for (int n = lane; n < P0; n += 32) s += Rr[n] * Tq[n];
  s = wsum(s);
  if (lane == 0) {
    rc[i] = s;
    rcf[i] = to_f(s);
  }
}

// The top of the tree in one stage each way.  T31 = T_1 T_2 maps the 16
// level-3 boxes under a level-1 box (index r = 4 q1 + q2, q1 the level-2
// quadrant, q2 the level-3 one; consecutive in Morton order) to its multipole,
// stored [n][u = r P_3 + m].  R1 = L2L_q (R T_0) maps the four level-1
// multipoles straight to the root's contribution to the local expansion of
// level-1 quadrant q, stored [q][n][u = q' P_1 + m], so that L(0) is never
// formed.  Both are read with lanes over u, along the multipoles as they lie in
// memory.  One thread per entry (consecutive threads along u), FP64 sums, with
// FP32 copies.
__global__ void m2m31_kernel(int P1, int P2, int P3, const cplx* __restrict__ m2m1, const cplx* __restrict__ m2m2,
                             cplx* __restrict__ c, cplxf* __restrict__ cf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int U = 16 * P3;
  if (i >= U * P1) return;
  const int n = i / U, u = i - n * U;
  const int r = u / P3, m = u - r * P3, q1 = r >> 2, q2 = r & 3;
  cplx s{0, 0};
  for (int k = 0; k < P2; ++k) s += m2m1[((size_t)q1 * P2 + k) * P1 + n] * m2m2[((size_t)q2 * P3 + m) * P2 + k];
  c[i] = s;
  cf[i] = to_f(s);
}

__global__ void root1_kernel(int P0, int P1, const cplx* __restrict__ l2l0, const cplx* __restrict__ rootc,
                          cplx* __restrict__ r1, cplxf* __restrict__ r1f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int U = 4 * P1;
  if (i >= 4 * P1 * U) return;
  const int qn = i / U, u = i - qn * U;
  const int q = qn / P1, n = qn - q * P1;
  cplx s{0, 0};
  for (int t = 0; t < P0; ++t) s += l2l0[((size_t)q * P0 + t) * P1 + n] * rootc[(size_t)u * P0 + t];
  r1[i] = s;
  r1f[i] = to_f(s);
}

// ------------------------------------------------------------ double-float sums
// A value h + l held as two FP32 numbers (about 48 bits).  acc += a b with
// a = ah + al, b = bh + bl: the product ah bh exactly as p + e (one rounding,
// its error by a fused multiply-add), the cross terms ah bl + al bh into e, and
// p added to acc.h by the two-sum of Knuth, whose error goes to acc.l with e.
// Explicitly rounded intrinsics keep the compiler from contracting the steps.
struct dflt {
  float h, l;
};

__device__ __forceinline__ void dd_mac(dflt& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  const float s = __fadd_rn(acc.h, p);
  const float v = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, v)), __fsub_rn(p, v));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

// acc += a b for complex a, b given as hi and lo parts
__device__ __forceinline__ void dd_cmac(dflt& re, dflt& im, cplxf ah, cplxf al, cplxf bh, cplxf bl) {
  dd_mac(re, ah.re, al.re, bh.re, bl.re);
  dd_mac(re, -ah.im, -al.im, bh.im, bl.im);
  dd_mac(im, ah.re, al.re, bh.im, bl.im);
  dd_mac(im, ah.im, al.im, bh.re, bl.re);
}

__device__ __forceinline__ dflt dd_add(dflt a, dflt b) {
  const float s = __fadd_rn(a.h, b.h);
  const float v = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
  return dflt{s, __fadd_rn(__fadd_rn(a.l, b.l), err)};
}

__device__ __forceinline__ dflt dd_wsum(dflt v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dflt w{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
    v = dd_add(v, w);
  }
  return v;
}

__device__ __forceinline__ double dd_value(dflt v) { return (double)v.h + (double)v.l; }

// Near-field sum of one target (sorted element s) in double-float arithmetic:
// the FP64 product's near field with FP32 instructions (GB300 issues FP64 at
// 1/64 of the FP32 rate) and FP64-level accuracy.  Writes the FP64 Un of s.
template <class C>
__device__ __forceinline__ void near_row_dd(const FusedArgs<C>& a, int s, int lane) {
  const longlong2 mt = __ldg(a.nr_meta + s);
  const int64_t r = mt.x;
  const int j0 = (int)(mt.y >> 32), ns = (int)(mt.y & 0xffffffffll);
  const cplxf* qh = a.nc_hi + r;
  const cplxf* ql = a.nc_lo + r;
  const cplxf* dh = a.dens_dd;
  const cplxf* dl = a.dens_dd + 2 * a.E;
  const int* src = a.nc_src + j0;
  dflt ur{0, 0}, ui{0, 0}, dr{0, 0}, di{0, 0};
  for (int j = lane; j < ns; j += 32) {
    const int f = src[j];
    const cplxf ph = ldcg(dh + 2 * f), pl = ldcg(dl + 2 * f), vh = ldcg(dh + 2 * f + 1), vl = ldcg(dl + 2 * f + 1);
    dd_cmac(ur, ui, qh[4 * j], ql[4 * j], ph, pl);
    dd_cmac(ur, ui, qh[4 * j + 1], ql[4 * j + 1], vh, vl);
    dd_cmac(dr, di, qh[4 * j + 2], ql[4 * j + 2], ph, pl);
    dd_cmac(dr, di, qh[4 * j + 3], ql[4 * j + 3], vh, vl);
  }
  ur = dd_wsum(ur);
  ui = dd_wsum(ui);
  dr = dd_wsum(dr);
  di = dd_wsum(di);
  if (lane == 0) {
    reinterpret_cast<cplx*>(a.Un)[2 * s] = cplx{dd_value(ur), dd_value(ui)};
    reinterpret_cast<cplx*>(a.Un)[2 * s + 1] = cplx{dd_value(dr), dd_value(di)};
  }
}

// Near-field sum of one target (sorted element s) from its leaf's cached
// [targets][sources] 2x2 blocks; lanes over the sources, two independent
// accumulator pairs.  Writes (U'_near, dU'_near) of s.
// Near-field sum of one target in differences (FP32 product): with the cached
// blocks B_sj of target s, sum_j B_sj psi_j = sum_j B_sj (psi_j - psi_s) + R_s psi_s.
// The densities are FP32 hi + lo pairs, so psi_j - psi_s keeps FP32 relative
// accuracy; R_s psi_s is added in FP64 by the L2P stage.  The hypersingular
// same-fiber blocks (entries ~1/h that cancel to O(1) on smooth densities) then
// lose no digits to the FP32 sums.
__device__ __forceinline__ void near_row_diff(const FusedArgs<cplxf>& a, int s, int lane) {
  // where the row lies (one load), the target's own densities, and the first
  // NJ source indices of every lane, all independent of one another
  const longlong2 mt = __ldg(a.nr_meta + s);
  const cplxf* row = a.nc_val + mt.x;
  const int* src = a.nc_src + (int)(mt.y >> 32);
  const int ns = (int)(mt.y & 0xffffffffll);
  const cplxf tph = ldcg(a.dens + 2 * s), tpl = ldcg(a.dlo + 2 * s);
  const cplxf tvh = ldcg(a.dens + 2 * s + 1), tvl = ldcg(a.dlo + 2 * s + 1);
  // NJ sources per lane and pass: their blocks and densities loaded together,
  // the next pass's source indices fetched meanwhile; a lane past the end takes
  // the target itself as its source, whose difference is zero
  constexpr int NJ = 4;
  int f[NJ];
#pragma unroll
  for (int k = 0; k < NJ; ++k) {
    const int jj = lane + 32 * k;
    f[k] = jj < ns ? __ldg(src + jj) : s;
  }
  cplxf u0{0, 0}, d0{0, 0}, u1{0, 0}, d1{0, 0};
  for (int jb = 0; jb < ns; jb += 32 * NJ) {
    cplxf p[NJ], v[NJ], q[NJ][4];
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
      const int jj = jb + lane + 32 * k;
      p[k] = (ldcg(a.dens + 2 * f[k]) - tph) + (ldcg(a.dlo + 2 * f[k]) - tpl);
      v[k] = (ldcg(a.dens + 2 * f[k] + 1) - tvh) + (ldcg(a.dlo + 2 * f[k] + 1) - tvl);
#pragma unroll
      for (int c = 0; c < 4; ++c) q[k][c] = jj < ns ? row[4 * jj + c] : cplxf{0, 0};
    }
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
      const int jj = jb + 32 * NJ + lane + 32 * k;
      f[k] = jj < ns ? __ldg(src + jj) : s;
    }
#pragma unroll
    for (int k = 0; k < NJ; k += 2) {
      u0 += q[k][0] * p[k] + q[k][1] * v[k];
      d0 += q[k][2] * p[k] + q[k][3] * v[k];
      u1 += q[k + 1][0] * p[k + 1] + q[k + 1][1] * v[k + 1];
      d1 += q[k + 1][2] * p[k + 1] + q[k + 1][3] * v[k + 1];
    }
  }
  const cplxf u = wsum(u0 + u1), du = wsum(d0 + d1);
  if (lane == 0) {
    a.Un[2 * s] = u;
    a.Un[2 * s + 1] = du;
  }
}

template <class C>
__device__ __forceinline__ void near_row(const FusedArgs<C>& a, int s, int lane) {
  if (a.nc_lo) {
    near_row_dd(a, s, lane);
    return;
  }
  if constexpr (sizeof(C) == sizeof(cplxf)) {
    if (a.dlo) {
      near_row_diff(a, s, lane);
      return;
    }
  }
  const longlong2 mt = __ldg(a.nr_meta + s);
  const C* row = a.nc_val + mt.x;
  const int* src = a.nc_src + (int)(mt.y >> 32);
  const int ns = (int)(mt.y & 0xffffffffll);
  C u0{0, 0}, d0{0, 0}, u1{0, 0}, d1{0, 0};
  int j = lane;
  for (; j + 32 < ns; j += 64) {
    const int f0 = src[j], f1 = src[j + 32];
    const C p0 = ldcg(a.dens + 2 * f0), v0 = ldcg(a.dens + 2 * f0 + 1);
    const C p1 = ldcg(a.dens + 2 * f1), v1 = ldcg(a.dens + 2 * f1 + 1);
    const C q0 = row[4 * j], q1 = row[4 * j + 1], q2 = row[4 * j + 2], q3 = row[4 * j + 3];
    const C r0 = row[4 * j + 128], r1 = row[4 * j + 129], r2 = row[4 * j + 130], r3 = row[4 * j + 131];
    u0 += q0 * p0 + q1 * v0;
    d0 += q2 * p0 + q3 * v0;
    u1 += r0 * p1 + r1 * v1;
    d1 += r2 * p1 + r3 * v1;
  }
  for (; j < ns; j += 32) {
    const int f = src[j];
    const C p = ldcg(a.dens + 2 * f), v = ldcg(a.dens + 2 * f + 1);
    u0 += row[4 * j] * p + row[4 * j + 1] * v;
    d0 += row[4 * j + 2] * p + row[4 * j + 3] * v;
  }
  const C u = wsum(u0 + u1), du = wsum(d0 + d1);
  if (lane == 0) {
    a.Un[2 * s] = u;
    a.Un[2 * s + 1] = du;
  }
}

// One piece of a near-field row in differences (FP32 product): at most
// NR_PIECE consecutive sources of target s, one pass of four sources per lane,
// added atomically into Un.  Pieces bound every near item's latency to one
// pass, whatever the row's length (crowded leaves give rows of ~600 sources).
// The descriptor d (read ahead by the stage loops) holds everything the piece
// needs to start: its block offset, its first source and (count, target).
constexpr int NR_PIECE = 128;
__device__ __forceinline__ void near_piece_diff(const FusedArgs<cplxf>& a, int4 d, int lane) {
  const int64_t r = (int64_t)(((unsigned long long)(unsigned)d.y << 32) | (unsigned)d.x);
  const int cnt = (int)((unsigned)d.w >> 24), s = (int)((unsigned)d.w & 0xffffffu);
  const cplxf* row = a.nc_val + r;
  const int* src = a.nc_src + d.z;
  const cplxf tph = ldcg(a.dens + 2 * s), tpl = ldcg(a.dlo + 2 * s);
  const cplxf tvh = ldcg(a.dens + 2 * s + 1), tvl = ldcg(a.dlo + 2 * s + 1);
  constexpr int NJ = NR_PIECE / 32;
  int f[NJ];
  cplxf q[NJ][4];
#pragma unroll
  for (int k = 0; k < NJ; ++k) {
    const int jj = lane + 32 * k;
    f[k] = jj < cnt ? __ldg(src + jj) : s;
#pragma unroll
    for (int c = 0; c < 4; ++c) q[k][c] = jj < cnt ? row[4 * jj + c] : cplxf{0, 0};
  }
  cplxf u0{0, 0}, d0{0, 0}, u1{0, 0}, d1{0, 0};
#pragma unroll
  for (int k = 0; k < NJ; k += 2) {
    const cplxf p0 = (ldcg(a.dens + 2 * f[k]) - tph) + (ldcg(a.dlo + 2 * f[k]) - tpl);
    const cplxf v0 = (ldcg(a.dens + 2 * f[k] + 1) - tvh) + (ldcg(a.dlo + 2 * f[k] + 1) - tvl);
    const cplxf p1 = (ldcg(a.dens + 2 * f[k + 1]) - tph) + (ldcg(a.dlo + 2 * f[k + 1]) - tpl);
    const cplxf v1 = (ldcg(a.dens + 2 * f[k + 1] + 1) - tvh) + (ldcg(a.dlo + 2 * f[k + 1] + 1) - tvl);
    u0 += q[k][0] * p0 + q[k][1] * v0;
    d0 += q[k][2] * p0 + q[k][3] * v0;
    u1 += q[k + 1][0] * p1 + q[k + 1][1] * v1;
    d1 += q[k + 1][2] * p1 + q[k + 1][3] * v1;
  }
  const cplxf u = wsum(u0 + u1), du = wsum(d0 + d1);
  if (lane == 0 && cnt > 0) {
    atomic_add(a.Un + 2 * s, u);
    atomic_add(a.Un + 2 * s + 1, du);
  }
}

// The near items [ifirst, nitem) of a stage that fall to one warp (every
// wstride-th from its first), item i being near item r0 + i - base: pieces
// (FP32 product in differences) with the next descriptor read while the current
// piece runs, so that a piece costs about two dependent loads instead of four;
// else whole rows.  nd: the warp's first descriptor, read by the caller before
// the stage's box items.
template <class C>
__device__ __forceinline__ void near_items(const FusedArgs<C>& a, int ifirst, int nitem, int wstride, int r0,
                                           int base, int4 nd, int lane) {
  if constexpr (sizeof(C) == sizeof(cplxf)) {
    if (a.npiece > 0) {
      for (int i = ifirst; i < nitem; i += wstride) {
        const int in = i + wstride;
        const int4 dn = in < nitem ? __ldg(a.nr_piece + r0 + (in - base)) : nd;
        near_piece_diff(a, nd, lane);
        nd = dn;
      }
      return;
    }
  }
  for (int i = ifirst; i < nitem; i += wstride) near_row(a, r0 + (i - base), lane);
}

// A warp's first near item of a stage (items from base on) and its descriptor.
template <class C>
__device__ __forceinline__ int first_near(const FusedArgs<C>& a, int wfirst, int wstride, int base, int nitem,
                                          int r0, int4* nd) {
  const int i0 = wfirst >= base ? wfirst : wfirst + ((base - wfirst + wstride - 1) / wstride) * wstride;
  *nd = int4{0, 0, 0, 0};
  if constexpr (sizeof(C) == sizeof(cplxf))
    if (a.npiece > 0 && i0 < nitem) *nd = __ldg(a.nr_piece + r0 + (i0 - base));
  return i0;
}

// Inverse block symbol of a regular-polygon fiber's whole same-fiber block of
// (I - A): the k1 part with the self terms (symbol fh, built above) plus the
// same-fiber k part, whose row pair is (i/4) (D, -i eta S) and c2 (i/4) (T,
// -i eta K) of the fiber's k table (Sec. 2: U, dU restricted to the fiber).
// The 2x2 symbol is inverted per frequency.  One block per fiber.
__global__ void precond_symbol_kernel(const int* __restrict__ fib_list, const int* __restrict__ foff,
                                      const int64_t* __restrict__ kbase, const cplx* __restrict__ kval,
                                      const int64_t* __restrict__ fh_base, const cplx* __restrict__ fh,
                                      double eta, cplx c2, const cplx* __restrict__ tw, cplx* __restrict__ pc,
                                      cplxf* __restrict__ pcf) {
  extern __shared__ __align__(128) unsigned char smraw[];
  cplx* sq = reinterpret_cast<cplx*>(smraw);      // [4][N]
  const int fb = fib_list[blockIdx.x];
  const int N = foff[fb + 1] - foff[fb], lg = __ffs(N) - 1;
  const cplx* kv = kval + 4 * kbase[fb];
  const cplx q4{0.0, 0.25};                       // i/4
  const cplx mie{0.0, -eta};                      // -i eta
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const cplx S = kv[4 * t], D = kv[4 * t + 1], K = kv[4 * t + 2], T = kv[4 * t + 3];
    sq[t] = q4 * D;
    sq[N + t] = q4 * (mie * S);
    sq[2 * N + t] = c2 * (q4 * T);
    sq[3 * N + t] = c2 * (q4 * (mie * K));
  }
  block_fft(sq, 4, lg, +1, tw);
  const cplx* B = fh + 4 * fh_base[fb];
  cplx* out = pc + 4 * fh_base[fb];
  cplxf* outf = pcf + 4 * fh_base[fb];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const cplx a = B[4 * k] + sq[k], b = B[4 * k + 1] + sq[N + k];
    const cplx c = B[4 * k + 2] + sq[2 * N + k], d = B[4 * k + 3] + sq[3 * N + k];
    const cplx det = a * d - b * c;
    const cplx id = cdiv(cplx{1, 0}, det);
    const cplx v[4] = {d * id, -(b * id), -(c * id), a * id};
    for (int j = 0; j < 4; ++j) {
      out[4 * k + j] = v[j];
      outf[4 * k + j] = to_f(v[j]);
    }
  }
}

// Preconditioner of a regular-polygon fiber whose element count is not a power
// of two: the same block-circulant inverse as above, kept as the row pair of
// its first element.  The 2x2 blocks b_d = k1 part (stored rows) + k part (k
// table) are transformed by a direct DFT, B(k) = sum_d b_d e^{2 pi i k d / N},
// inverted per frequency, and transformed back, c_d = (1/N) sum_k B(k)^-1
// e^{-2 pi i k d / N}; rows[r][2d + s] = c_d^(r,s).  One block per fiber.
__global__ void precond_rows_kernel(const int* __restrict__ fib_list, const int* __restrict__ foff,
                                    const int64_t* __restrict__ fb_base, const cplx* __restrict__ fbrows,
                                    const int64_t* __restrict__ kbase, const cplx* __restrict__ kval, double eta,
                                    cplx c2, const int64_t* __restrict__ pr_base, cplx* __restrict__ pr,
                                    cplxf* __restrict__ prf) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const int fb = fib_list[blockIdx.x];
  const int N = foff[fb + 1] - foff[fb];
  cplx* b = reinterpret_cast<cplx*>(smraw);        // [4][N] blocks b_d
  cplx* bh = b + 4 * (size_t)N;                    // [4][N] B(k)^-1
  cplx* om = bh + 4 * (size_t)N;                   // [N] e^{2 pi i j / N}
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * j / N, &sn, &cs);
    om[j] = cplx{cs, sn};
  }
  const cplx* R = fbrows + fb_base[fb];
  const cplx* kv = kval + 4 * kbase[fb];
  const cplx q4{0.0, 0.25}, mie{0.0, -eta};
  for (int d = threadIdx.x; d < N; d += blockDim.x) {
    const cplx S = kv[4 * d], D = kv[4 * d + 1], K = kv[4 * d + 2], T = kv[4 * d + 3];
    b[d] = R[2 * d] + q4 * D;
    b[N + d] = R[2 * d + 1] + q4 * (mie * S);
    b[2 * N + d] = R[2 * N + 2 * d] + c2 * (q4 * T);
    b[3 * N + d] = R[2 * N + 2 * d + 1] + c2 * (q4 * (mie * K));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    cplx a[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int d = 0, kd = 0; d < N; ++d) {          // kd = k d mod N
      const cplx w = om[kd];
      for (int j = 0; j < 4; ++j) a[j] += b[j * N + d] * w;
      kd += k;
      if (kd >= N) kd -= N;
    }
    const cplx det = a[0] * a[3] - a[1] * a[2];
    const cplx id = cdiv(cplx{1, 0}, det);
    bh[k] = a[3] * id;
    bh[N + k] = -(a[1] * id);
    bh[2 * N + k] = -(a[2] * id);
    bh[3 * N + k] = a[0] * id;
  }
  __syncthreads();
  cplx* out = pr + pr_base[fb];
  cplxf* outf = prf + pr_base[fb];
  for (int d = threadIdx.x; d < N; d += blockDim.x) {
    cplx c[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int k = 0, kd = 0; k < N; ++k) {          // e^{-2 pi i k d / N} = conj(om[k d mod N])
      const cplx w = conj(om[kd]);
      for (int j = 0; j < 4; ++j) c[j] += bh[j * N + k] * w;
      kd += d;
      if (kd >= N) kd -= N;
    }
    const double inv = 1.0 / N;
    const cplx v[4] = {inv * c[0], inv * c[1], inv * c[2], inv * c[3]};
    out[2 * d] = v[0];
    out[2 * d + 1] = v[1];
    out[2 * N + 2 * d] = v[2];
    out[2 * N + 2 * d + 1] = v[3];
    outf[2 * d] = to_f(v[0]);
    outf[2 * d + 1] = to_f(v[1]);
    outf[2 * N + 2 * d] = to_f(v[2]);
    outf[2 * N + 2 * d + 1] = to_f(v[3]);
  }
}

// y = P^{-1} x (original order, FP64 in and out, arithmetic in C): per fiber,
// y^(r) = IFFT( sum_s Binv^(r,s) FFT(x^(s)) ) where a symbol exists, y = x
// elsewhere.  One block per fiber.
template <class C>
__device__ void precond_fiber(int fb, const int* __restrict__ foff, const int64_t* __restrict__ fh_base,
                              const C* __restrict__ pc, const C* __restrict__ tw, const int64_t* __restrict__ pr_base,
                              const C* __restrict__ pr, const cplx* __restrict__ x, cplx* __restrict__ y, C* xs) {
  const int f0 = foff[fb], N = foff[fb + 1] - f0;
  const int64_t base = fh_base[fb];
  if (base < 0) {
    const int64_t rb = pr_base ? pr_base[fb] : -1;
    if (rb < 0) {
      for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) y[2 * f0 + t] = x[2 * f0 + t];
      return;
    }
    // block-circulant inverse from its row pair: y[2e + r] = sum_c R_r[c] x[(c + 2e) mod 2N]
    const int n2 = 2 * N;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) xs[t] = from_d<C>(x[2 * f0 + t]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const C* R0 = pr + rb;
    const C* R1 = R0 + n2;
    for (int r = 2 * warp; r < n2; r += 2 * nw) {
      C a0{0, 0}, a1{0, 0};
      for (int c = lane; c < n2; c += 32) {
        int i = c + r;
        if (i >= n2) i -= n2;
        const C xv = xs[i];
        a0 += R0[c] * xv;
        a1 += R1[c] * xv;
      }
      a0 = wsum(a0);
      a1 = wsum(a1);
      if (lane == 0) {
        y[2 * f0 + r] = to_d(a0);
        y[2 * f0 + r + 1] = to_d(a1);
      }
    }
    return;
  }
  const int lg = __ffs(N) - 1;
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int q = t >> lg, f = t & (N - 1);
    xs[t] = from_d<C>(x[2 * (f0 + f) + q]);
  }
  block_fft(xs, 2, lg, -1, tw);
  const C* Bi = pc + 4 * base;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const C x0 = xs[k], x1 = xs[N + k];
    const C* bk = Bi + 4 * k;
    xs[k] = bk[0] * x0 + bk[1] * x1;
    xs[N + k] = bk[2] * x0 + bk[3] * x1;
  }
  block_fft(xs, 2, lg, +1, tw);
  const double inv = 1.0 / N;
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
    const int r = t >> lg, e = f0 + (t & (N - 1));
    y[2 * e + r] = inv * to_d(xs[t]);
  }
}

// y = P^-1 x, one block per fiber (see precond_fiber).
template <class C>
__global__ void precond_apply_kernel(int M, const int* __restrict__ foff, const int64_t* __restrict__ fh_base,
                                     const C* __restrict__ pc, const C* __restrict__ tw,
                                     const int64_t* __restrict__ pr_base, const C* __restrict__ pr,
                                     const cplx* __restrict__ x, cplx* __restrict__ y, const int* done,
                                     int tws_off) {
  if (done && *(volatile const int*)done != 0) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  C* xs = reinterpret_cast<C*>(smraw);
  C* tws = xs + tws_off;                          // twiddles in shared memory
  for (int i = threadIdx.x; i < 512; i += blockDim.x) tws[i] = tw[i];
  __syncthreads();
  precond_fiber<C>(blockIdx.x, foff, fh_base, pc, tws, pr_base, pr, x, y, xs);
}

// ------------------------------------------------------------ device-side GMRES step
// One Arnoldi step of GMRES after w = A z_j, as one cooperative launch with two
// device-wide barriers: classical Gram-Schmidt applied twice (h1 = V^H w,
// w -= V h1, h2 = V^H w, w -= V h2), v_{j+1} = w / ||w||, and then, by one
// thread, the Givens rotations
// of the new Hessenberg column h1 + h2 (+ ||w|| below the diagonal), the
// rotated right-hand side g and the residual estimate |g_{j+1}| / ||b||.  The
// step raises the cycle's done flag when the estimate reaches the threshold,
// on breakdown (||w|| = 0) or at the restart length; every kernel of the
// cycle queued after that returns at once.  Each block owns one
// contiguous slice of the n entries; the dot products go one warp per basis
// column over the slice and meet by atomic adds.  The sums of step j live in
// accumulator set j mod 2, and step j clears the other set for step j + 1.
// The norm of the final w comes from the second pass: with V orthonormal,
// ||w - V h2||^2 = ||w||^2 - ||h2||^2, and after the first pass h2 is of the
// order of the rounding error, so the difference loses no accuracy.  The last
// update w -= V h2 is then done where v_{j+1} is written (fiber by fiber with
// the preconditioner) and needs no barrier of its own.  The dot products and
// the updates run in C, the precision of the products: FP32 for the inner
// solves of the mixed-precision refinement, whose tolerance (never below 1e-4
// relative) lies far above FP32 rounding, so the FP64 pipe (1/64 of the FP32 rate
// on this GPU) carries none of them; the basis, the Hessenberg matrix, the
// rotations and the sums across blocks stay FP64.
struct ArnArgs {
  int n, m, j;
  cplx* V;                           // [(m+1)][n] orthonormal basis
  cplx* w;                           // [n] A z_j on entry
  cplx* H;                           // [(m+1)][m] Hessenberg matrix, rotated into triangular form
  cplx* cs;                          // [m] Givens rotations
  cplx* sn;
  cplx* g;                           // [m+1] rotated right-hand side (beta e_1 at the cycle start)
  cplx* acc;                         // [2][2 (m+1) + 1] CGS2 sums h1, h2 and ||w||^2, by step parity
  double* ctl;                       // [0] estimate (out), [1] ||b||, [2] threshold
  int* ictl;                         // [0] done, [1] steps completed in the cycle, [2] reason (1 est, 2 breakdown, 3 restart)
  unsigned long long* bar;
  int* err;
  // with the block-Jacobi preconditioner, z_{j+1} = P^-1 v_{j+1} fiber by fiber
  cplx* Zn;                          // [n] z_{j+1}, or null (no preconditioner)
  int M;
  const int* foff;
  const int64_t* fh_base;
  const void* pc;                    // inverse symbols (FFT fibers), in the precision of the products
  const void* tw;
  const int64_t* pr_base;            // circulant inverse row pairs (the other regular polygons)
  const void* pr;
  int tws_off;                       // shared-memory offset (in C) of the twiddle copy
};

constexpr int ARN_MAXC = 256;        // columns of the basis the kernel can hold (restart length <= 250)

template <class C>
__device__ __forceinline__ void arn_dots(const ArnArgs& a, int nc, int t0, int t1, cplx* out, int warp, int lane) {
  for (int c = warp; c < nc; c += FW) {
    const cplx* v = a.V + (size_t)c * a.n;
    C s{0, 0};
#pragma unroll 4
    for (int t = t0 + lane; t < t1; t += 32) s += conj(from_d<C>(v[t])) * from_d<C>(a.w[t]);
    s = wsum(s);
    if (lane == 0) atomic_add(out + c, to_d(s));
  }
}

// EXT: the rotations of the serial part are staged in the dynamic shared memory
// (at least 2 ARN_MAXC complex values) instead of a static array of their own.
template <class C, bool EXT>
__device__ __forceinline__ bool arnoldi_body(const ArnArgs& a, const int b, const int G, unsigned long long limit) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ cplx sh[ARN_MAXC];
  __shared__ C shc[ARN_MAXC];                       // sh in the precision of the updates
  __shared__ double red[FW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t0 = (int)((int64_t)a.n * b / G), t1 = (int)((int64_t)a.n * (b + 1) / G);
  const int nc = a.j + 1, S = 2 * (a.m + 1) + 1;
  cplx* h1 = a.acc + (size_t)(a.j & 1) * S;
  cplx* h2 = h1 + (a.m + 1);
  double* nrm = reinterpret_cast<double*>(h2 + (a.m + 1));
  if (b == 0) {
    cplx* other = a.acc + (size_t)((a.j + 1) & 1) * S;
    for (int i = threadIdx.x; i < S; i += FB) other[i] = cplx{0, 0};
  }
  // h1 = V^H w
  arn_dots<C>(a, nc, t0, t1, h1, warp, lane);
  if (!group_barrier(a.bar, a.err, limit, G, b)) return false;
  // w -= V h1; ||w||^2; h2 = V^H w
  for (int i = threadIdx.x; i < nc; i += FB) shc[i] = from_d<C>(ldcg(h1 + i));
  __syncthreads();
  double part = 0;
  for (int t = t0 + threadIdx.x; t < t1; t += FB) {
    C v = from_d<C>(a.w[t]);
#pragma unroll 4
    for (int c = 0; c < nc; ++c) v -= from_d<C>(a.V[(size_t)c * a.n + t]) * shc[c];
    const cplx vd = to_d(v);
    a.w[t] = vd;
    part += vd.re * vd.re + vd.im * vd.im;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
    for (int i = 0; i < FW; ++i) tot += red[i];
    atomicAdd(nrm, tot);
  }
  arn_dots<C>(a, nc, t0, t1, h2, warp, lane);
  if (!group_barrier(a.bar, a.err, limit, G, b)) return false;
  // ||w - V h2||^2 = ||w||^2 - ||h2||^2; v_{j+1} = (w - V h2) / ||w - V h2|| and,
  // with the preconditioner, z_{j+1} = P^-1 v_{j+1} (one block per fiber: a
  // fiber's block of P^-1 reads only its own entries)
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += FB) {
    sh[i] = ldcg(h2 + i);
    shc[i] = from_d<C>(sh[i]);
  }
  __syncthreads();
  double s2 = 0;
  for (int c = 0; c < nc; ++c) s2 += sh[c].re * sh[c].re + sh[c].im * sh[c].im;
  const double hn = sqrt(fmax(*(volatile double*)nrm - s2, 0.0));
  const double inv = hn > 0 ? 1.0 / hn : 0.0;
  cplx* vn = a.V + (size_t)(a.j + 1) * a.n;
  if (a.Zn) {
    C* xs = reinterpret_cast<C*>(smraw);
    C* tws = xs + a.tws_off;                        // twiddles in shared memory
    if (b < a.M) {
      for (int i = threadIdx.x; i < 512; i += FB) tws[i] = static_cast<const C*>(a.tw)[i];
    }
    for (int fb = b; fb < a.M; fb += G) {
      __syncthreads();
      for (int t = 2 * a.foff[fb] + threadIdx.x; t < 2 * a.foff[fb + 1]; t += FB) {
        C v = from_d<C>(a.w[t]);
#pragma unroll 4
        for (int c = 0; c < nc; ++c) v -= from_d<C>(a.V[(size_t)c * a.n + t]) * shc[c];
        vn[t] = inv * to_d(v);
      }
      __syncthreads();
      precond_fiber<C>(fb, a.foff, a.fh_base, static_cast<const C*>(a.pc), tws, a.pr_base,
                       static_cast<const C*>(a.pr), vn, a.Zn, xs);
    }
  } else {
    for (int t = t0 + threadIdx.x; t < t1; t += FB) {
      C v = from_d<C>(a.w[t]);
#pragma unroll 4
      for (int c = 0; c < nc; ++c) v -= from_d<C>(a.V[(size_t)c * a.n + t]) * shc[c];
      vn[t] = inv * to_d(v);
    }
  }
  if (b == G - 1) {
    // the new column of H and its Givens rotations (by the last block, which
    // has no fiber to precondition when the fibers are fewer than the blocks);
    // the operands are staged in shared memory first, so that the serial part
    // runs without global-memory latency
    const int j = a.j, m = a.m;
    cplx* col = sh;                                   // [j + 2]
    cplx* rot;                                        // cs, sn of the earlier steps
    if constexpr (EXT) {
      rot = reinterpret_cast<cplx*>(smraw);
    } else {
      __shared__ cplx rot_s[2 * ARN_MAXC];
      rot = rot_s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += FB) col[i] = ldcg(h1 + i) + ldcg(h2 + i);
    for (int i = threadIdx.x; i < j; i += FB) {
      rot[i] = a.cs[i];
      rot[ARN_MAXC + i] = a.sn[i];
    }
    if (threadIdx.x == 0) col[j + 1] = cplx{hn, 0};
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < j; ++i) {
        const cplx x0 = col[i], x1 = col[i + 1], c = rot[i], sn = rot[ARN_MAXC + i];
        col[i] = conj(c) * x0 + conj(sn) * x1;
        col[i + 1] = (-sn) * x0 + c * x1;
      }
      const cplx x0 = col[j], x1 = col[j + 1];
      const double den = sqrt(x0.re * x0.re + x0.im * x0.im + x1.re * x1.re + x1.im * x1.im);
      cplx c{1, 0}, sn{0, 0};
      if (den != 0) {
        c = (1.0 / den) * x0;
        sn = (1.0 / den) * x1;
      }
      a.cs[j] = c;
      a.sn[j] = sn;
      col[j] = conj(c) * x0 + conj(sn) * x1;
      col[j + 1] = cplx{0, 0};
      const cplx gj = a.g[j];
      a.g[j] = conj(c) * gj;
      const cplx gn = (-sn) * gj;
      a.g[j + 1] = gn;
      const double est = sqrt(gn.re * gn.re + gn.im * gn.im) / a.ctl[1];
      a.ctl[0] = est;
      a.ictl[1] = j + 1;
      const int reason = est <= a.ctl[2] ? 1 : (hn == 0 ? 2 : (j + 1 == m ? 3 : 0));
      if (reason) {
        a.ictl[2] = reason;
        a.ictl[0] = 1;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += FB) a.H[(size_t)i * m + j] = col[i];
  }
  return true;
}

template <class C>
__global__ void __launch_bounds__(FB) arnoldi_kernel(const __grid_constant__ ArnArgs a) {
  if (*(volatile const int*)a.ictl != 0) return;
  arnoldi_body<C, false>(a, (int)blockIdx.x, (int)gridDim.x, 1000000000ull);
}

// y = R^{-1} g over the steps completed in the cycle (R: the rotated H) by
// back substitution: R (up to 32 steps) is staged in shared memory by the
// block, then one thread solves.  Called by all threads of one block.
// EXT: R and g staged in the dynamic shared memory (at least 1056 complex
// values) instead of static arrays of their own.
template <bool EXT>
__device__ void arn_backsolve(const cplx* __restrict__ H, const cplx* __restrict__ g, int m, int jf,
                              cplx* __restrict__ y) {
  constexpr int RS = 32;
  cplx *R, *gs;
  if constexpr (EXT) {
    extern __shared__ __align__(128) unsigned char smraw[];
    R = reinterpret_cast<cplx*>(smraw);
    gs = R + RS * RS;
  } else {
    __shared__ cplx R_s[RS * RS], gs_s[RS];
    R = R_s;
    gs = gs_s;
  }
  const bool staged = jf <= RS;
  __syncthreads();
  if (staged) {
    for (int t = threadIdx.x; t < jf * jf; t += blockDim.x) {
      const int i = t / jf, q = t - i * jf;
      R[i * RS + q] = H[(size_t)i * m + q];
    }
    for (int t = threadIdx.x; t < jf; t += blockDim.x) gs[t] = g[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx ys[RS];
    for (int i = jf - 1; i >= 0; --i) {
      cplx v = staged ? gs[i] : g[i];
      if (staged) {
        for (int q = i + 1; q < jf; ++q) v -= R[i * RS + q] * ys[q];
        ys[i] = cdiv(v, R[i * RS + i]);
        y[i] = ys[i];
      } else {
        for (int q = i + 1; q < jf; ++q) v -= H[(size_t)i * m + q] * y[q];
        y[i] = cdiv(v, H[(size_t)i * m + i]);
      }
    }
  }
  __syncthreads();
}

__global__ void arnoldi_solve_kernel(const cplx* __restrict__ H, const cplx* __restrict__ g, int m,
                                     const int* __restrict__ ictl, cplx* __restrict__ y) {
  arn_backsolve<false>(H, g, m, ictl[1], y);
}

// Warp items: item i goes to block i mod nb and, within the block, to warp
// (i / nb + i mod nb) mod nw(), so that a stage whose item count is not a
// multiple of the grid spreads its extra items over all four sub-partitions
// of the SMs instead of piling them on warp 0.  Returns the first item of
// warp w of block b; the stride is nb * nw().
__device__ __forceinline__ int warp_first(int b, int w, int nb) {
  return b + nb * ((w - b % nw() + nw()) % nw());
}

// Rows rb..re of one fiber's same-fiber block (FP32 product) in differences:
// with the element t of rows (r, r+1) and x_t its two unknowns,
//   y_r = sum_c R_r[c] (x_c - x_t^(c mod 2)) + sum_{c even} R_r[c] x_t^(0) + sum_{c odd} R_r[c] x_t^(1),
// the first sum in FP32 on hi + lo copies of x (differences to FP32 relative
// accuracy, no cancellation of the hypersingular entries), the row sums
// (FP64, from frs) times x_t in FP64.  xs holds the hi parts [n2] and the lo
// parts [n2].
__device__ void fiber_rows_diff(const FusedArgs<cplxf>& a, cplxf* xs, int fb, int rb, int re, int f0, int n2,
                                bool cir, int warp, int lane) {
  cplxf* xl = xs + n2;
  __syncthreads();
  for (int i = threadIdx.x; i < n2; i += nt()) {
    const cplx v = a.x[2 * f0 + i];
    xs[i] = to_f(v);
    xl[i] = split_lo(v);
  }
  __syncthreads();
  for (int r = rb + 2 * warp; r < re; r += 2 * nw()) {
    const cplxf* row0 = a.fb_val + a.fb_base[fb] + (cir ? 0 : (int64_t)r * n2);
    const cplxf* row1 = row0 + n2;
    const int sh = cir ? r : 0;
    const bool two = r + 1 < re;
    // every column this lane visits has the lane's parity
    const cplxf th = xs[r + (lane & 1)], tl = xl[r + (lane & 1)];
    cplxf a0{0, 0}, b0v{0, 0};
    for (int c = lane; c < n2; c += 32) {
      int i0 = c + sh;
      if (i0 >= n2) i0 -= n2;
      const cplxf d = (xs[i0] - th) + (xl[i0] - tl);
      a0 += row0[c] * d;
      if (two) b0v += row1[c] * d;
    }
    const cplxf s0 = wsum(a0);
    const cplxf s1 = wsum(b0v);
    if (lane == 0) {
      const cplx x0 = a.x[2 * f0 + r], x1 = a.x[2 * f0 + r + 1];
      const cplx* R = a.frs + 2 * (size_t)(2 * f0 + r);
      a.y[2 * f0 + r] = to_d(s0) + R[0] * x0 + R[1] * x1;
      if (two) a.y[2 * f0 + r + 1] = to_d(s1) + R[2] * x0 + R[3] * x1;
    }
  }
}

// The FFT-applied fibers of the same-fiber part (block b0 of nb), in the
// arithmetic of F: y^(r) = IFFT(sum_s B^(r,s) FFT(x^(s))), one block per fiber;
// xs holds [2N] values of F and, from tws_off on, the twiddle table.
template <class F>
__device__ void fiber_fft(int nfft, const int* fft_fib, const int* foff, const int64_t* fh_base, const F* fh_val,
                          const F* tw, const cplx* x, cplx* y, F* xs, int tws_off, int b0, int nb) {
  using R = decltype(F{}.re);
  // the twiddle table in shared memory: the FFT passes then wait on no global load
  F* tws = xs + tws_off;
  if (b0 < nfft) {
    for (int i = threadIdx.x; i < 512; i += nt()) tws[i] = tw[i];
  }
  for (int b = b0; b < nfft; b += nb) {
    const int fb = fft_fib[b];
    const int f0 = foff[fb], N = foff[fb + 1] - f0, lg = __ffs(N) - 1;
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * N; t += nt()) {
      const int q = t >> lg, f = t & (N - 1);
      xs[t] = from_d<F>(x[2 * (f0 + f) + q]);
    }
    block_fft(xs, 2, lg, -1, tws);
    const F* Bh = fh_val + 4 * fh_base[fb];
    for (int k = threadIdx.x; k < N; k += nt()) {
      const F x0 = xs[k], x1 = xs[N + k];
      const F* bk = Bh + 4 * k;
      xs[k] = bk[0] * x0 + bk[1] * x1;
      xs[N + k] = bk[2] * x0 + bk[3] * x1;
    }
    block_fft(xs, 2, lg, +1, tws);
    const R inv = (R)1 / (R)N;
    for (int t = threadIdx.x; t < 2 * N; t += nt()) {
      const int rr = t >> lg, e = f0 + (t & (N - 1));
      y[2 * e + rr] = to_d(inv * xs[t]);
    }
  }
}

// The same-fiber blocks of eq. 9 (the k1 part with the self terms, and for a
// regular polygon also the k part) applied to x, written to y in the
// original element order; block b0 of nb blocks.  A regular-polygon fiber
// whose element count is a power of two goes by FFT (one block per fiber),
// y^(r) = IFFT(sum_s B^(r,s) FFT(x^(s))); the others by cached rows (one block
// per chunk of 32 rows; a circulant block is read from its generating row
// pair with x rotated by 2e).
template <class C>
__device__ void fiber_part(const FusedArgs<C>& a, C* xs, int b0, int nb, int warp, int lane) {
  // the FP32 product's FFTs run in FP64 when its FP64 symbols are given: the
  // block symbol of the hypersingular operator grows with the frequency, so FP32
  // rounding of a smooth density's high modes would be amplified
  if constexpr (sizeof(C) == sizeof(cplxf)) {
    if (a.fh64) {
      fiber_fft<cplx>(a.nfft, a.fft_fib, a.foff, a.fh_base, a.fh64, a.tw64, a.x, a.y, reinterpret_cast<cplx*>(xs),
                      a.tws_off, b0, nb);
    } else {
      fiber_fft<C>(a.nfft, a.fft_fib, a.foff, a.fh_base, a.fh_val, a.tw, a.x, a.y, xs, a.tws_off, b0, nb);
    }
  } else {
    fiber_fft<C>(a.nfft, a.fft_fib, a.foff, a.fh_base, a.fh_val, a.tw, a.x, a.y, xs, a.tws_off, b0, nb);
  }
  for (int b = b0; b < a.nchunk; b += nb) {
    const int fb = a.fb_chunk[3 * b], rb = a.fb_chunk[3 * b + 1], re = a.fb_chunk[3 * b + 2];
    const int f0 = a.foff[fb], n2 = 2 * (a.foff[fb + 1] - f0);
    const bool cir = a.circ[fb] != 0;
    if constexpr (sizeof(C) == sizeof(cplxf)) {
      if (a.frs) {
        fiber_rows_diff(a, xs, fb, rb, re, f0, n2, cir, warp, lane);
        continue;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n2; i += nt()) xs[i] = from_d<C>(a.x[2 * f0 + i]);
    __syncthreads();
    for (int r = rb + 2 * warp; r < re; r += 2 * nw()) {
      const C* row0 = a.fb_val + a.fb_base[fb] + (cir ? 0 : (int64_t)r * n2);
      const C* row1 = row0 + n2;
      const int sh = cir ? r : 0;
      const bool two = r + 1 < re;
      C a0{0, 0}, a1{0, 0}, b0v{0, 0}, b1v{0, 0};
      int c = lane;
      for (; c + 32 < n2; c += 64) {
        int i0 = c + sh, i1 = c + 32 + sh;
        if (i0 >= n2) i0 -= n2;
        if (i1 >= n2) i1 -= n2;
        const C x0 = xs[i0], x1 = xs[i1];
        a0 += row0[c] * x0;
        a1 += row0[c + 32] * x1;
        if (two) {
          b0v += row1[c] * x0;
          b1v += row1[c + 32] * x1;
        }
      }
      for (; c < n2; c += 32) {
        int i0 = c + sh;
        if (i0 >= n2) i0 -= n2;
        a0 += row0[c] * xs[i0];
        if (two) b0v += row1[c] * xs[i0];
      }
      const C s0 = wsum(a0 + a1);
      const C s1 = wsum(b0v + b1v);
      if (lane == 0) {
        a.y[2 * f0 + r] = to_d(s0);
        if (two) a.y[2 * f0 + r + 1] = to_d(s1);
      }
    }
  }
}

// M2M into the nbi boxes of level l as block items: group g of nw() boxes (one
// per warp) goes to the block of rank g mod G, which stages the four stacked quadrant
// operators [4 Pc][P] once (the same for every box of the level) and applies
// them to each warp's box in one pass over its 4 Pc child coefficients.  A few
// blocks then carry the level while the others go on to their warp items.
// Called by all threads of the block.
template <class C>
__device__ void m2m_quad(const FusedArgs<C>& a, int l, int nbi, C* sT, C* wsm, int warp, int lane, int rb,
                         bool have, unsigned long long* dg, int G) {
  const int ng = (nbi + nw() - 1) / nw();
  if (rb >= ng) return;
  const int P = a.P[l], Pc = a.P[l + 1], K = 4 * Pc;
  const int S = a.S[l], O = a.O[l], Sc = a.S[l + 1], Oc = a.O[l + 1];
  if (!have) {           // not staged ahead, at the end of the previous stage
    __syncthreads();
    stage_copy_quad(sT, a.m2m[l] + (size_t)Oc * S + O, P, Pc, S, Sc);
  }
  __syncthreads();
  if (dg && threadIdx.x == 0) dg[8192] = gtimer();     // diagnostic: operators staged
  for (int g = rb; g < ng; g += G) {
    const int i = g * nw() + warp;
    if (i >= nbi) continue;
    const int box = a.ne[l][i];
    // the four children's multipoles (those of empty boxes are kept at zero),
    // every load issued before the first store
    __syncwarp();
    for (int t0 = 0; t0 < K; t0 += 160) {
      constexpr int KU = 5;
      C v[KU];
#pragma unroll
      for (int k = 0; k < KU; ++k) {
        const int t = t0 + lane + 32 * k, q = t / Pc;
        v[k] = t < K ? ldcg(a.M[l + 1] + (size_t)(4 * box + q) * Sc + Oc + (t - q * Pc)) : C{0, 0};
      }
#pragma unroll
      for (int k = 0; k < KU; ++k)
        if (t0 + lane + 32 * k < K) wsm[t0 + lane + 32 * k] = v[k];
    }
    __syncwarp();
    if (dg && threadIdx.x == 0) dg[16384] = gtimer();    // diagnostic: children gathered
    C* Mo = a.M[l] + (size_t)box * S + O;
    warp_colmv(sT, P, wsm, K, lane, [&](int n, C v) { Mo[n] = v; });
  }
}

// L2L into group g of nw() boxes of level l (box g nw() + warp), the four stacked
// quadrant operators [4 Pp][P] already staged in sT; each box applies the block
// of its own quadrant to its parent's local expansion.
template <class C>
__device__ __forceinline__ void l2l_quad_group(const FusedArgs<C>& a, int l, int nl2l, int g, const C* sT, C* wsm,
                                               int warp, int lane) {
  const int i = g * nw() + warp;
  if (i >= nl2l) return;
  const int P = a.P[l], Pp = a.P[l - 1];
  const int S = a.S[l], O = a.O[l], Sp = a.S[l - 1], Op = a.O[l - 1];
  const int box = a.ne[l][i], par = box >> 2, q = box & 3;
  __syncwarp();
  for (int m = lane; m < Pp; m += 32) wsm[m] = ldcg(a.L[l - 1] + (size_t)par * Sp + Op + m);
  __syncwarp();
  C* Lo = a.L[l] + (size_t)box * S + O;
  warp_colmv(sT + (size_t)q * Pp * P, P, wsm, Pp, lane, [&](int n, C v) { atomic_add(Lo + n, v); });
}

// M2M into the nbi boxes of level l with the quadrant operators T_q (stored
// [q][m child][n parent]) staged in shared memory one after another: warp item i
// (the warp's box) accumulates its four children's contributions over the four
// quadrant phases.  All threads of the block call this (block-level barriers);
// a block with no box in a round leaves the loop, which is uniform over it.
// ---------------------------------------------------------------- tensor-core M2L
// TMEM columns a block holds while the product runs (>= the largest tc_kp).
constexpr int TC_NCOL = 128;

// Bounded wait for the completion of the MMAs committed to mbar in phase ph.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t ph, unsigned long long limit) {
  const uint32_t addr = tc::smem_u32(mbar);
  unsigned long long t0 = 0;
  for (int spin = 0;; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(ph)
        : "memory");
    if (done) return true;
    if ((spin & 15) == 15) {
      const unsigned long long t = gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit) return false;
    }
  }
}

// Largest MMA N = K of the single-launch product's tensor-core M2L: A and B
// then take 3 x 128 x 80 + 3 x 80 x 80 BF16 values (97.5 KB of shared memory).
constexpr int TC_KPMAX = 80;

__host__ __device__ constexpr size_t tc_smem_bytes(int kp) {
  return (size_t)3 * tc::TILE * kp * 2 + (size_t)3 * kp * kp * 2;
}

// M2L of one block item at level l: tile = 128 target boxes (rows of the MMA),
// and a group of the offsets present in the tile.  For each offset o, thread 0
// starts the bulk copy of B = T_o (three BF16 parts, canonical layout, built at
// set-up) into shared memory while the block writes A: row t holds
// alpha^m M(src_t) with K index 2c / 2c + 1 for the real / imaginary part of
// coefficient c, in three BF16 parts.  Thread 0 then issues the six split
// products of order <= 2,
//   A0B0 + A0B1 + A1B0 + A0B2 + A1B1 + A2B0,
// accumulated in FP32 in tensor memory over the group's offsets (about FP32
// accuracy).  B's output rows hold the real parts of the target coefficients
// at 0 .. P - 1 and the imaginary parts from tc::imrow(P) on, so the epilogue
// reads both in aligned groups of 8 columns and adds them into L (atomically:
// L2L and the tile's other groups add into the same boxes).  Called by all
// threads; false when a wait ran out (after a second bounded wait for what was
// in flight).
__device__ bool tc_m2l_item(const FusedArgs<cplxf>& a, int l, int item, unsigned char* smraw, uint32_t tmem,
                            uint64_t* mbar, uint32_t& phase, int warp, int lane) {
  using bf = __nv_bfloat16;
  const int kp = a.tc_kp[l], P = a.P[l], S = a.S[l], O = a.O[l];
  const int ngrp = a.tc_ngrp[l];
  const int tile = item / ngrp, grp = item - tile * ngrp;
  const int ntot = a.tc_noff[l][tile];
  const int og = (ntot + ngrp - 1) / ngrp, o0 = grp * og, o1 = min(ntot, o0 + og);
  if (o0 >= o1) return true;
  bf* sA = reinterpret_cast<bf*>(smraw);                 // 3 x 128 x kp
  bf* sB = sA + 3 * tc::TILE * kp;                        // 3 x kp x kp
  const uint32_t bbytes = (uint32_t)(3 * kp * kp * 2);
  // nq threads per row of A (the block's threads over the 128 rows)
  const int t = threadIdx.x, row = t & (tc::TILE - 1), part = t >> 7, nq = nt() >> 7;
  const uint32_t idesc = tc::idesc_bf16(tc::TILE, kp), sbo = (uint32_t)(kp / 8) * 128;
  uint64_t* mb_mma = mbar;
  uint64_t* mb_b = mbar + 1;
  __shared__ int s_fail;
  // each offset's accumulator is read back into registers and summed there in
  // FP32 (round to nearest), so that the tensor memory accumulates one offset's
  // split products only: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of
  // the tile), the warps of one lane quarter taking turns over the groups of 8
  // coefficients (at most TC_CH groups each; P <= 40)
  constexpr int TC_CH = 2;
  const int lq = warp & 3, ch = warp >> 2, nch = nw() >> 2;
  const int nc8 = (P + 7) / 8, im0 = tc::imrow(P);
  const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
  float accr[TC_CH][8], acci[TC_CH][8];
#pragma unroll
  for (int k = 0; k < TC_CH; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) accr[k][j] = acci[k][j] = 0.f;
  // earlier generic-proxy writes of this shared memory (other items, stages)
  // are ordered before the bulk copies and MMAs of the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  for (int oi = o0; oi < o1; ++oi) {
    const int o = a.tc_offs[l][tile * 49 + oi];
    if (t == 0) {
      const bf* gB = reinterpret_cast<const bf*>(a.tc_B[l]) + (size_t)o * 3 * kp * kp;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mb_b)), "r"(bbytes)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       tc::smem_u32(sB)),
                   "l"(gB), "r"(bbytes), "r"(tc::smem_u32(mb_b))
                   : "memory");
    }
    {
      const size_t ti = ((size_t)tile * 49 + oi) * tc::TILE + row;
      const int src = a.tc_src[l][ti];
      const cplxf ph = from_d<cplxf>(phase_m(a.alpha, src >= 0 ? a.tc_img[l][ti] : 0));
      const cplxf* Ms = a.M[l] + (size_t)(src >= 0 ? src : 0) * S + O;
      // this thread's groups g = part + nq j of 8 components (4 coefficients);
      // all loads first
      constexpr int GJ = TC_KPMAX / 16;
      cplxf v[GJ][4];
#pragma unroll
      for (int j = 0; j < GJ; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int g = part + nq * j, c = 4 * g + q;
          v[j][q] = (src >= 0 && 8 * g < kp && c < P) ? ldcg(Ms + c) : cplxf{0, 0};
        }
#pragma unroll
      for (int j = 0; j < GJ; ++j) {
        const int g = part + nq * j;
        if (8 * g < kp) {
          uint32_t w0[4], w1[4], w2[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const cplxf z = ph * v[j][q];
            bf a0, a1, a2, b0, b1, b2;
            tc::split3(z.re, a0, a1, a2);
            tc::split3(z.im, b0, b1, b2);
            w0[q] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(b0) << 16);
            w1[q] = (uint32_t)__bfloat16_as_ushort(a1) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
            w2[q] = (uint32_t)__bfloat16_as_ushort(a2) | ((uint32_t)__bfloat16_as_ushort(b2) << 16);
          }
          const uint32_t off = tc::canon(row, 8 * g, kp) >> 4;    // 16-byte units
          reinterpret_cast<uint4*>(sA)[off] = make_uint4(w0[0], w0[1], w0[2], w0[3]);
          reinterpret_cast<uint4*>(sA + tc::TILE * kp)[off] = make_uint4(w1[0], w1[1], w1[2], w1[3]);
          reinterpret_cast<uint4*>(sA + 2 * tc::TILE * kp)[off] = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        }
      }
    }
    // the generic-proxy writes of A become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      int f = 0;
      if (!mbar_wait(mb_b, phase, a.wait_ns)) {
        f = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int pa[6] = {0, 0, 1, 0, 1, 2};
        const int pb[6] = {0, 1, 0, 2, 1, 0};
        for (int q = 0; q < 6; ++q) {
          const uint32_t abase = tc::smem_u32(sA + pa[q] * tc::TILE * kp);
          const uint32_t bbase = tc::smem_u32(sB + pb[q] * kp * kp);
          for (int kk = 0; kk < kp / 16; ++kk) {
            const uint64_t ad = tc::sdesc(abase + kk * 256, 128, sbo);
            const uint64_t bd = tc::sdesc(bbase + kk * 256, 128, sbo);
            const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc::smem_u32(mb_mma))
                     : "memory");
      }
      s_fail = f;
    }
    __syncthreads();
    if (s_fail) {
      // no MMA was issued; the bulk copy may still be running
      if (t == 0) {
        mbar_wait(mb_b, phase, a.wait_ns);
        atomicExch(a.err, 1);
      }
      __syncthreads();
      return false;
    }
    // every thread waits for the MMAs (their operands are overwritten next)
    const bool ok = mbar_wait(mb_mma, phase, a.wait_ns);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        mbar_wait(mb_mma, phase, a.wait_ns);
        atomicExch(a.err, 1);
      }
      __syncthreads();
      return false;
    }
    phase ^= 1u;
    // this offset's accumulator into the registers (the next offset's first
    // MMA, issued after a block barrier, overwrites it)
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int k = 0; k < TC_CH; ++k) {
      const int c8 = ch + nch * k;
      if (c8 < nc8) {
        uint32_t vr[8], vi[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]),
                       "=r"(vr[7])
                     : "r"(lane_addr + 8 * c8));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]),
                       "=r"(vi[7])
                     : "r"(lane_addr + im0 + 8 * c8));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          accr[k][j] += __uint_as_float(vr[j]);
          acci[k][j] += __uint_as_float(vi[j]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // epilogue: the row's sums into L
  {
    const int r = lq * 32 + lane;
    const int tgt = a.tc_box[l][tile * tc::TILE + r];
    cplxf* Lt = a.L[l] + (size_t)(tgt >= 0 ? tgt : 0) * S + O;
    if (tgt >= 0) {
#pragma unroll
      for (int k = 0; k < TC_CH; ++k) {
        const int c8 = ch + nch * k;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = 8 * c8 + j;
          if (c8 < nc8 && c < P) atomic_add(Lt + c, cplxf{accr[k][j], acci[k][j]});
        }
      }
    }
  }
  // the next item's first MMA overwrites the accumulator: every read is done
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

// Block items of the next stage, so that a block can stage their operators in
// shared memory at the end of the current stage (off the next stage's critical
// path): the M2M quadrant stack of a B stage, the first M2L chunk's operator and
// the L2L quadrant stack of a D stage.  The rules are those of the stages.
template <class C>
__device__ __forceinline__ bool bstage_quad(const FusedArgs<C>& a, int l, int wstride, int* ng) {
  const int P = a.P[l], Pc = a.P[l + 1];
  const bool top = (int64_t)a.nne[l] * P <= wstride;
  const bool quad = sizeof(C) == sizeof(cplxf) && l >= 1 && !top && 4 * Pc <= PF_NCOEF && 4 * Pc * P <= a.treg;
  *ng = quad ? (a.nne[l] + nw() - 1) / nw() : 0;
  return quad;
}
struct DItems {
  bool ql2l;
  int ntc, nchu, ngl, nl2l;
};
template <class C, bool TC>
__device__ __forceinline__ DItems dstage_items(const FusedArgs<C>& a, int l, int wstride) {
  const int P = a.P[l], Pp = a.P[l - 1];
  const bool top = (int64_t)a.nne[l] * P <= wstride;
  DItems d;
  d.nl2l = top ? a.nne[l] * P : a.nne[l];
  const bool wpair = a.m2l_warp || P > TSP;
  d.ql2l = sizeof(C) == sizeof(cplxf) && !top && Pp <= PF_NCOEF && 4 * Pp * P <= (a.tregL > 0 ? a.tregL : a.treg);
  const bool tcl = TC && sizeof(C) == sizeof(cplxf) && a.tc_kp[l] > 0;
  d.ntc = tcl ? a.tc_ntile[l] * a.tc_ngrp[l] : 0;
  d.nchu = (wpair || tcl) ? 0 : a.nch[l];
  d.ngl = d.ql2l ? (d.nl2l + nw() - 1) / nw() : 0;
  return d;
}
// The M2L chunk b's operator of level l, staged transposed ([target][source]).
template <class C>
__device__ __forceinline__ void stage_chunk(const FusedArgs<C>& a, int l, int b, C* sT) {
  const int P = a.P[l], S = a.S[l], O = a.O[l];
  const C* To = a.m2lt[l] + (size_t)a.ch_off[l][b] * S * S + (size_t)O * S + O;   // [n source][l target]
  if (S == P)
    stage_copy(sT, To, P * P, IdxTranspose{P});
  else
    stage_copy_bt(sT, To, P, S);
}
template <class C>
__device__ __forceinline__ void stage_l2l_quad(const FusedArgs<C>& a, int l, C* dst) {
  stage_copy_quad(dst, a.l2l[l - 1] + (size_t)a.O[l - 1] * a.S[l] + a.O[l], a.P[l], a.P[l - 1], a.S[l], a.S[l - 1]);
}

template <class C>
__device__ void m2m_staged(const FusedArgs<C>& a, int l, int nbi, int wfirst, int wstride, C* sT, C* wsm, int lane,
                           int bid) {
  const int P = a.P[l], Pc = a.P[l + 1], PP = Pc * P;
  const int S = a.S[l], O = a.O[l], Sc = a.S[l + 1], Oc = a.O[l + 1];
  const bool dd = a.m2ml[l] != nullptr;
  const int rounds = (nbi + wstride - 1) / wstride;
  for (int rd = 0; rd < rounds; ++rd) {
    if (bid + rd * wstride >= nbi) break;
    const int i = wfirst + rd * wstride;
    const bool mine = i < nbi;
    const int box = mine ? a.ne[l][i] : 0;
    cplxf* wh = reinterpret_cast<cplxf*>(wsm);
    cplxf* wl = wh + PF_NCOEF;
    __syncwarp();
    if (mine) {
      for (int t = lane; t < 4 * Pc; t += 32) {
        const int q = t / Pc, ch = 4 * box + q;
        const C v = a.bb[l + 1][ch] < a.be[l + 1][ch] ? ldcg(a.M[l + 1] + (size_t)ch * Sc + Oc + (t - q * Pc))
                                                      : C{0, 0};
        if (dd) {
          const cplx d = to_d(v);
          wh[t] = cplxf{(float)d.re, (float)d.im};
          wl[t] = split_lo(d);
        } else {
          wsm[t] = v;
        }
      }
    }
    C acc[2] = {C{0, 0}, C{0, 0}};
    dflt re[2] = {{0, 0}, {0, 0}}, im[2] = {{0, 0}, {0, 0}};
    for (int q = 0; q < 4; ++q) {
      __syncthreads();
      // the used [Pc][P] block of T_q: source rows q Sc + Oc + m, target columns O + n
      if (dd) {
        cplxf* th = reinterpret_cast<cplxf*>(sT);
        stage_copy(th, a.m2mh[l] + (size_t)(q * Sc + Oc) * S + O, PP, IdxBlock{P, S});
        stage_copy(th + PP, a.m2ml[l] + (size_t)(q * Sc + Oc) * S + O, PP, IdxBlock{P, S});
      } else {
        stage_copy(sT, a.m2m[l] + (size_t)(q * Sc + Oc) * S + O, PP, IdxBlock{P, S});
      }
      __syncthreads();
      if (!mine) continue;
      for (int h = 0; h < 2; ++h) {
        const int n = lane + 32 * h;
        if (n >= P) break;
        if (dd) {
          const cplxf* th = reinterpret_cast<const cplxf*>(sT);
#pragma unroll 4
          for (int m = 0; m < Pc; ++m)
            dd_cmac(re[h], im[h], th[m * P + n], th[PP + m * P + n], wh[q * Pc + m], wl[q * Pc + m]);
        } else {
          C s0{0, 0}, s1{0, 0};
          int m = 0;
#pragma unroll 4
          for (; m + 1 < Pc; m += 2) {
            s0 += sT[m * P + n] * wsm[q * Pc + m];
            s1 += sT[(m + 1) * P + n] * wsm[q * Pc + m + 1];
          }
          if (m < Pc) s0 += sT[m * P + n] * wsm[q * Pc + m];
          acc[h] += s0 + s1;
        }
      }
    }
    if (mine) {
      for (int h = 0; h < 2; ++h) {
        const int n = lane + 32 * h;
        if (n >= P) break;
        a.M[l][(size_t)box * S + O + n] = dd ? from_d<C>(cplx{dd_value(re[h]), dd_value(im[h])}) : acc[h];
      }
    }
  }
  __syncthreads();
}

// L2L into the nl2l boxes of level l, quadrant operators (stored [q][m parent]
// [n child]) staged in shared memory; each warp's box takes the phase of its
// own quadrant.  Called by all threads of the block, like m2m_staged.
template <class C>
__device__ void l2l_staged(const FusedArgs<C>& a, int l, int nl2l, int wfirst, int wstride, C* sT, C* wsm, int lane,
                           int bid) {
  const int P = a.P[l], Pp = a.P[l - 1], PP = Pp * P;
  const int S = a.S[l], O = a.O[l], Sp = a.S[l - 1], Op = a.O[l - 1];
  // FP64 product: double-float arithmetic from the hi and lo tables
  const bool dd = a.l2ll[l - 1] != nullptr;
  const int rounds = (nl2l + wstride - 1) / wstride;
  cplxf* wh = reinterpret_cast<cplxf*>(wsm);
  cplxf* wl = wh + PF_NCOEF;
  for (int rd = 0; rd < rounds; ++rd) {
    if (bid + rd * wstride >= nl2l) break;
    const int i = wfirst + rd * wstride;
    const bool mine = i < nl2l;
    const int box = mine ? a.ne[l][i] : 0, par = box >> 2, qb = box & 3;
    __syncwarp();
    if (mine)
      for (int m = lane; m < Pp; m += 32) {
        const C v = ldcg(a.L[l - 1] + (size_t)par * Sp + Op + m);
        if (dd) {
          const cplx d = to_d(v);
          wh[m] = cplxf{(float)d.re, (float)d.im};
          wl[m] = split_lo(d);
        } else {
          wsm[m] = v;
        }
      }
    for (int q = 0; q < 4; ++q) {
      __syncthreads();
      // the used [Pp][P] block of T_q: source rows q Sp + Op + m, target columns O + n
      if (dd) {
        cplxf* th = reinterpret_cast<cplxf*>(sT);
        stage_copy(th, a.l2lh[l - 1] + (size_t)(q * Sp + Op) * S + O, PP, IdxBlock{P, S});
        stage_copy(th + PP, a.l2ll[l - 1] + (size_t)(q * Sp + Op) * S + O, PP, IdxBlock{P, S});
      } else {
        stage_copy(sT, a.l2l[l - 1] + (size_t)(q * Sp + Op) * S + O, PP, IdxBlock{P, S});
      }
      __syncthreads();
      if (!mine || qb != q) continue;
      for (int n = lane; n < P; n += 32) {
        if (dd) {
          const cplxf* th = reinterpret_cast<const cplxf*>(sT);
          dflt re{0, 0}, im{0, 0};
#pragma unroll 4
          for (int m = 0; m < Pp; ++m) dd_cmac(re, im, th[m * P + n], th[PP + m * P + n], wh[m], wl[m]);
          atomic_add(a.L[l] + (size_t)box * S + O + n, from_d<C>(cplx{dd_value(re), dd_value(im)}));
          continue;
        }
        C s0{0, 0}, s1{0, 0};
        int m = 0;
#pragma unroll 4
        for (; m + 1 < Pp; m += 2) {
          s0 += sT[m * P + n] * wsm[m];
          s1 += sT[(m + 1) * P + n] * wsm[m + 1];
        }
        if (m < Pp) s0 += sT[m * P + n] * wsm[m];
        atomic_add(a.L[l] + (size_t)box * S + O + n, s0 + s1);
      }
    }
  }
  __syncthreads();
}

// Register budget: three resident blocks of 256 threads per SM for the FP64
// product, two for the FP32 one (the counts launch_fused runs them at).  The
// tensor-core form (TC, FP32 only) holds tensor memory, with which the device
// keeps one block per SM: it runs 512 threads per block instead.
template <class C, bool TC>
__device__ __forceinline__ bool fused_body(const FusedArgs<C>& a, const int bid, const int G) {
  extern __shared__ __align__(128) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wfirst = warp_first(bid, warp, G), wstride = G * nw();
  C* wsm = sm + a.treg + a.tregL + (size_t)warp * PF_NCOEF;     // per-warp scratch
  C* sT = sm;                                                   // [P][P] staged M2L operator (row stride P, odd)
  C* sL = sm + a.treg;                                          // staged L2L quadrant stack (when tregL > 0)
  const int D = a.D;
  int ks = 0;
  // block items of consecutive stages start at blocks half a grid apart, so the
  // blocks that stage the next stage's operators at the end of this one are not
  // the ones carrying this stage's block items; rank(stage) is the block's rank
  // in a stage's block-item order
  auto rank = [&](int stage) { return (int)((bid + G - ((stage & 1) ? G / 2 : 0)) % G); };
  int pf_b = -1, pf_c = -1, pf_cl = -1, pf_l = -1;   // what is staged ahead: B level, chunk (level), L2L level
  // at the end of a stage, before its barrier: stage the operators of this
  // block's first block items of the next stage (index sn), a B stage of level
  // lb or a D stage of level ld (-1: none)
  auto prefetch = [&](int sn, int lb, int ld) {
    const int rb = rank(sn);
    if (lb >= 1) {
      int ng = 0;
      if (bstage_quad(a, lb, wstride, &ng) && rb < ng) {
        __syncthreads();
        stage_copy_quad(sT, a.m2m[lb] + (size_t)a.O[lb + 1] * a.S[lb] + a.O[lb], a.P[lb], a.P[lb + 1], a.S[lb],
                        a.S[lb + 1]);
        pf_b = lb;
      }
    } else if (ld >= 1) {
      const DItems d = dstage_items<C, TC>(a, ld, wstride);
      if (d.ntc > 0) return;                    // tensor-core items take the whole shared memory
      bool synced = false;
      if (rb < d.nchu) {
        __syncthreads();
        synced = true;
        stage_chunk(a, ld, rb, sT);
        pf_c = rb;
        pf_cl = ld;
      }
      const int first = d.nchu, b0 = rb >= first ? rb : rb + ((first - rb + G - 1) / G) * G;
      if (a.tregL > 0 && d.ngl > 0 && b0 < first + d.ngl) {
        if (!synced) __syncthreads();
        stage_l2l_quad(a, ld, sL);
        pf_l = ld;
      }
    }
  };
  // FP32 product with tensor-core M2L levels: the block holds TC_NCOL columns
  // of tensor memory and two mbarriers (MMA completion, operator copy) for the
  // whole launch; tc_leave gives the columns back on every way out
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  uint32_t tc_phase = 0;
  bool tc_on = false;
  if constexpr (TC && sizeof(C) == sizeof(cplxf)) {
    if (a.tc_any) {
      if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                     "r"(TC_NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
      }
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tc_on = true;
    }
  }
  auto tc_leave = [&]() {
    if constexpr (TC && sizeof(C) == sizeof(cplxf)) {
      if (tc_on) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0)
          asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(TC_NCOL) : "memory");
      }
    }
  };
  stage_stamp(a.stamp, ks++, bid);

  // ------------------------------------------------------------ A: gather + P2M, clear L; fiber part
  {
    for (int l = 1; l <= D; ++l) {
      C* Lz = a.L[l];
      const size_t nz = (size_t)a.nbox[l] * a.S[l];
      for (size_t t = (size_t)bid * nt() + threadIdx.x; t < nz; t += (size_t)G * nt()) Lz[t] = C{0, 0};
    }
    if (sizeof(C) == sizeof(cplxf) && a.npiece > 0)      // the near pieces add into Un
      for (size_t t = (size_t)bid * nt() + threadIdx.x; t < 2 * (size_t)a.E; t += (size_t)G * nt())
        a.Un[t] = C{0, 0};
    // blocks [gA, G) apply the same-fiber blocks while the others run P2M
    const int gA = G - a.fblk;
    if (bid < gA) {
      const int PD = a.P[D];
      for (int i = warp_first(bid, warp, gA); i < a.nne[D]; i += gA * nw()) {
        const int box = a.ne[D][i], s0 = a.bb[D][box], s1 = a.be[D][box];
        // the leaf's elements GU x 32 at a time: indices and phases, then the
        // inputs, each batch of loads issued before its first use
        constexpr int GU = sizeof(C) == sizeof(cplxf) ? 4 : 2;
        for (int sb = s0; sb < s1; sb += 32 * GU) {
          int ei[GU];
          cplx pk[GU], xa[GU], xb[GU];
#pragma unroll
          for (int k = 0; k < GU; ++k) {
            const int s = sb + lane + 32 * k;
            ei[k] = s < s1 ? a.perm[s] : 0;
            pk[k] = s < s1 ? a.ph[s] : cplx{0, 0};
          }
#pragma unroll
          for (int k = 0; k < GU; ++k) {
            xa[k] = a.x[2 * ei[k]];
            xb[k] = a.x[2 * ei[k] + 1];
          }
#pragma unroll
          for (int k = 0; k < GU; ++k) {
          const int s = sb + lane + 32 * k;
          if (s < s1) {
            const cplx p = pk[k];
            const cplx e0 = p * xa[k], e1 = p * xb[k];     // FP64, then rounded
            a.dens[2 * s] = from_d<C>(e0);
            a.dens[2 * s + 1] = from_d<C>(e1);
            if (a.dens_dd) {
              a.dens_dd[2 * s] = cplxf{(float)e0.re, (float)e0.im};
              a.dens_dd[2 * s + 1] = cplxf{(float)e1.re, (float)e1.im};
              a.dens_dd[2 * a.E + 2 * s] = split_lo(e0);
              a.dens_dd[2 * a.E + 2 * s + 1] = split_lo(e1);
            }
            if (a.dlo) {
              a.dlo[2 * s] = split_lo(e0);
              a.dlo[2 * s + 1] = split_lo(e1);
            }
          }
          }
        }
        __syncwarp();
        if (a.p2ml) {
          // FP64 product in double-float arithmetic, from the densities' hi and
          // lo parts just written by this warp
          const cplxf* dh = a.dens_dd;
          const cplxf* dl = a.dens_dd + 2 * a.E;
          for (int n = lane; n < PD; n += 32) {
            dflt re{0, 0}, im{0, 0};
            for (int f = s0; f < s1; ++f) {
              const size_t c0 = (size_t)f * 2 * PD + n, c1 = c0 + PD;
              dd_cmac(re, im, a.p2mh[c0], a.p2ml[c0], dh[2 * f], dl[2 * f]);
              dd_cmac(re, im, a.p2mh[c1], a.p2ml[c1], dh[2 * f + 1], dl[2 * f + 1]);
            }
            a.M[D][(size_t)box * PD + n] = from_d<C>(cplx{dd_value(re), dd_value(im)});
          }
          continue;
        }
        const int SD = a.S[D], OD = a.O[D];
        // coefficients n < 32 (PD & ~31) a lane each over all the leaf's
        // elements; the last PD mod 32 split over lane groups that share the
        // elements, their sums combined by shuffles
        const int full = PD & ~31;
        for (int n0 = 0; n0 < full; n0 += 32) {
          const int n = n0 + lane;
          C acc0{0, 0}, acc1{0, 0};
#pragma unroll 8
          for (int f = s0; f < s1; ++f) {
            const C* cf = a.p2m + (size_t)f * 2 * SD + OD;
            acc0 += cf[n] * a.dens[2 * f];
            acc1 += cf[SD + n] * a.dens[2 * f + 1];
          }
          a.M[D][(size_t)box * SD + OD + n] = acc0 + acc1;
        }
        if (PD > full) {
          const int r = PD - full, g = 32 / r, grp = lane / r, nr = lane - grp * r;
          const int n = full + nr;
          C acc0{0, 0}, acc1{0, 0};
          if (grp < g) {
#pragma unroll 4
            for (int f = s0 + grp; f < s1; f += g) {
              const C* cf = a.p2m + (size_t)f * 2 * SD + OD;
              acc0 += cf[n] * a.dens[2 * f];
              acc1 += cf[SD + n] * a.dens[2 * f + 1];
            }
          }
          const C acc = acc0 + acc1;
          C sum = acc;
          for (int k = 1; k < g; ++k) {
            const C o = shfl_c(acc, k * r + nr);
            sum += o;
          }
          if (lane < r) a.M[D][(size_t)box * SD + OD + n] = sum;
        }
      }
    }
    if (a.fblk == 0)
      fiber_part(a, sm, bid, G, warp, lane);
    else if (bid >= gA)
      fiber_part(a, sm, bid - gA, a.fblk, warp, lane);
    // the first B stage's (or D_1's) operators, staged ahead; the fiber part
    // is done with the shared memory
    {
      const int lst = a.top3 ? 2 : 0;
      __syncthreads();
      if (D - 1 >= lst)
        prefetch(ks, D - 1, -1);
      else
        prefetch(ks, -1, 1);
    }
  }
  if (!group_barrier(a.bar, a.err, a.wait_ns, G, bid, a.arrive ? a.arrive + (size_t)(ks - 1) * G : nullptr)) {
      tc_leave();
      return false;
    }
  stage_stamp(a.stamp, ks++, bid);

  // ------------------------------------------------------------ B: M2M (+ root)
  // the last B stage: level 2 when it also forms M(1), else the root
  // the near-field rows need only the densities of stage A: they are spread
  // evenly over all B and D stages, whose FMM work leaves most warps idle
  const int lstop = a.top3 ? 2 : 0, nbst = D - lstop, nst = nbst + D;
  // near items: pieces of rows (FP32 product) or whole rows
  const int NI = (sizeof(C) == sizeof(cplxf) && a.npiece > 0) ? a.npiece : a.E;
  for (int l = D - 1; l >= lstop; --l) {
    const int P = a.P[l], Pc = a.P[l + 1];
    const int jst = D - 1 - l;
    const int r0 = a.near_first ? (jst == 0 ? 0 : NI) : (int)((int64_t)NI * jst / nst);
    const int r1 = a.near_first ? NI : (int)((int64_t)NI * (jst + 1) / nst);
    // near the top of the tree the boxes are too few to occupy the grid: one
    // warp per output coefficient, lanes over the 4 Pc child coefficients.  The
    // root then forms L(0) = (R T_0) [M(1) of its four children] at once.
    const bool top = (int64_t)a.nne[l] * P <= wstride;
    const int nbi = top ? a.nne[l] * P : a.nne[l];
    // with top3, the level-2 stage adds M(1) (one warp per coefficient, from the
    // 16 level-3 boxes below)
    const int nx = (a.top3 && l == 2) ? a.nne[1] * a.P[1] : 0;
    const int nitem = nbi + nx + (r1 - r0);
    // boxes of the larger levels: the block stages each quadrant operator in
    // shared memory once and applies it to all of its warps' boxes (a warp on
    // its own would stream the whole [4][Pc][P] table from L2 for every box)
    const bool quad = sizeof(C) == sizeof(cplxf) && l >= 1 && !top && 4 * Pc <= PF_NCOEF && 4 * Pc * P <= a.treg;
    const bool staged = quad || (l >= 1 && !top && 4 * Pc <= PF_NCOEF && Pc * P <= TSIZE && P <= 64);
    if (quad) {
      m2m_quad(a, l, nbi, sT, wsm, warp, lane, rank(ks - 1), pf_b == l,
               a.bdone ? a.bdone + (size_t)(ks - 1) * G + bid : nullptr, G);
      pf_b = -1;
    }
    else if (staged)
      m2m_staged(a, l, nbi, wfirst, wstride, sT, wsm, lane, bid);
    if (a.bdone && threadIdx.x == 0) a.bdone[(size_t)(ks - 1) * G + bid] = gtimer();
    int4 nd;
    const int inear = first_near(a, wfirst, wstride, nbi + nx, nitem, r0, &nd);
    for (int i = wfirst; i < nbi + nx; i += wstride) {
      if (staged && i < nbi) continue;
      if (i >= nbi) {
        // M(1) of a level-1 box from its 16 level-3 boxes; the multipoles of
        // empty level-3 boxes are kept at zero, so the sum runs without branches
        const int k = i - nbi, P1 = a.P[1], P3 = a.P[3], S3 = a.S[3], O3 = a.O[3];
        const int U1 = 16 * S3;
        const int b1 = a.ne[1][k / P1], n = k % P1;
        const C* A = a.m2m31 + (size_t)(a.O[1] + n) * U1 + O3;
        const C* M3 = a.M[3] + (size_t)b1 * U1 + O3;
        C acc{0, 0};
#pragma unroll 4
        for (int u = lane; u < 16 * P3; u += 32) {
          const int r = u / P3, v = r * S3 + (u - r * P3);
          acc += A[v] * ldcg(M3 + v);
        }
        acc = wsum(acc);
        if (lane == 0) a.M[1][(size_t)b1 * a.S[1] + a.O[1] + n] = acc;
        continue;
      }
      if (top) {
        const int bi = i / P, n = i - bi * P;
        const int box = a.ne[l][bi];
        const int S = a.S[l], Sc = a.S[l + 1], Oc = a.O[l + 1];
        C acc{0, 0};
        if (l == 0) {
          // L(0) of root box from the level-1 multipoles of every root (R T_0
          // folded; rows (level-1 box, coefficient), columns (root, coefficient))
          const int RS = a.nroot * S;
          const C* A = a.rootc + (size_t)box * S + a.O[0] + n;
          for (int u = lane; u < 4 * a.nroot * Pc; u += 32) {
            const int ch = u / Pc, m = u - ch * Pc;
            if (a.bb[1][ch] < a.be[1][ch])
              acc += A[(size_t)(ch * Sc + Oc + m) * RS] * ldcg(a.M[1] + (size_t)ch * Sc + Oc + m);
          }
        } else {
          const C* A = a.m2m[l] + a.O[l] + n;
          for (int u = lane; u < 4 * Pc; u += 32) {
            const int q = u / Pc, m = u - q * Pc, ch = 4 * box + q;
            if (a.bb[l + 1][ch] < a.be[l + 1][ch])
              acc += A[(size_t)(q * Sc + Oc + m) * S] * ldcg(a.M[l + 1] + (size_t)ch * Sc + Oc + m);
          }
        }
        acc = wsum(acc);
        if (lane == 0) {
          if (l == 0)
            a.L[0][(size_t)box * S + a.O[0] + n] = acc;
          else
            a.M[l][(size_t)box * S + a.O[l] + n] = acc;
        }
        continue;
      }
      const int box = a.ne[l][i];
      if (a.m2ml[l] && 4 * Pc <= PF_NCOEF) {
        // FP64 product in double-float arithmetic: the four children's
        // multipoles split into hi and lo parts, the operator from its tables
        cplxf* wh = reinterpret_cast<cplxf*>(wsm);
        cplxf* wl = wh + PF_NCOEF;
        __syncwarp();
        for (int t = lane; t < 4 * Pc; t += 32) {
          const int q = t / Pc, ch = 4 * box + q;
          const cplx v = a.bb[l + 1][ch] < a.be[l + 1][ch] ? to_d(ldcg(a.M[l + 1] + (size_t)ch * Pc + (t - q * Pc)))
                                                           : cplx{0, 0};
          wh[t] = cplxf{(float)v.re, (float)v.im};
          wl[t] = split_lo(v);
        }
        __syncwarp();
        for (int n = lane; n < P; n += 32) {
          dflt re{0, 0}, im{0, 0};
#pragma unroll 4
          for (int u = 0; u < 4 * Pc; ++u)
            dd_cmac(re, im, a.m2mh[l][(size_t)u * P + n], a.m2ml[l][(size_t)u * P + n], wh[u], wl[u]);
          a.M[l][(size_t)box * P + n] = from_d<C>(cplx{dd_value(re), dd_value(im)});
        }
      } else {
        // the generic form (the FP32 product may run at orders below its
        // tables': the used coefficients and operator blocks sit at offsets O
        // in rows of S): the children one quadrant at a time
        const int S = a.S[l], O = a.O[l], Sc = a.S[l + 1], Oc = a.O[l + 1];
        for (int n0 = 0; n0 < P; n0 += 32) {
          const int n = n0 + lane;
          C acc{0, 0};
          for (int q = 0; q < 4; ++q) {
            const int ch = 4 * box + q;
            if (a.bb[l + 1][ch] >= a.be[l + 1][ch]) continue;
            __syncwarp();
            for (int m = lane; m < Pc; m += 32) wsm[m] = ldcg(a.M[l + 1] + (size_t)ch * Sc + Oc + m);
            __syncwarp();
            if (n < P) acc += colmv(a.m2m[l] + (size_t)(q * Sc + Oc) * S + O + n, S, wsm, Pc);
          }
          if (n < P) a.M[l][(size_t)box * S + O + n] = acc;
        }
      }
      if (l == 0) {
        // root: L(0) = R M(0), the images |m| >= 2 through the lattice sums
        // (only on a grid too small for the coefficient-per-warp form above)
        const int S = a.S[0], O = a.O[0];
        __syncwarp();
        for (int m = lane; m < P; m += 32) wsm[m] = ldcg(a.M[0] + O + m);
        __syncwarp();
        for (int t = lane; t < P; t += 32) {
          C r{0, 0};
          for (int m = 0; m < P; ++m) r += a.root[(size_t)(O + t) * S + O + m] * wsm[m];
          a.L[0][O + t] = r;
        }
      }
    }
    near_items(a, inear, nitem, wstride, r0, nbi + nx, nd, lane);
    // the next stage's operators, staged ahead (this stage's items are done
    // with the shared memory once the block has passed this point)
    if (l - 1 >= lstop)
      prefetch(ks, l - 1, -1);
    else
      prefetch(ks, -1, 1);
    if (!group_barrier(a.bar, a.err, a.wait_ns, G, bid, a.arrive ? a.arrive + (size_t)(ks - 1) * G : nullptr)) {
      tc_leave();
      return false;
    }
    stage_stamp(a.stamp, ks++, bid);
  }

  // ------------------------------------------------------------ D: L2L + M2L
  for (int l = 1; l <= D; ++l) {
    const int P = a.P[l], Pp = a.P[l - 1];
    // L2L: one warp per output coefficient while the boxes are few, else one
    // warp per box
    const bool top = (int64_t)a.nne[l] * P <= wstride;
    const int nl2l = top ? a.nne[l] * P : a.nne[l];
    // M2L one warp per pair (operator rows through L1/L2), or one block per
    // chunk of pairs sharing the offset (operator staged in shared memory)
    const bool wpair = a.m2l_warp || P > TSP;
    // L2L as block items (groups of nw() boxes, the stacked quadrant operators
    // staged once per block) when the FP32 tables fit the staging region
    // M2L on the tensor cores at this level (FP32 product): block items over
    // (tile of 128 targets, group of offsets) in place of the chunks
    const DItems di = dstage_items<C, TC>(a, l, wstride);
    const bool ql2l = di.ql2l, tcl = di.ntc > 0;
    const int ntc = di.ntc, nchu = di.nchu, ngl = di.ngl;
    // block items: the tensor-core tiles or the staged M2L chunks first, then
    // the L2L groups (in their own region when there is one); then the warp items
    {
      C* sLL = a.tregL > 0 ? sL : sT;
      bool l2l_ready = pf_l == l;
      const int rb = rank(ks - 1);
      for (int b0 = rb; b0 < ntc + nchu + ngl; b0 += G) {
        if (b0 < ntc) {
          if constexpr (TC && sizeof(C) == sizeof(cplxf)) {
            // a wait that ran out has set the error flag: the next barrier ends the product
            if (!tc_m2l_item(a, l, b0, smraw, s_tmem, s_mbar, tc_phase, warp, lane)) break;
          }
          continue;
        }
        const int b = b0 - ntc;
        if (b >= nchu) {
          if (!l2l_ready) {
            __syncthreads();                                  // sT of the last chunk is done
            stage_l2l_quad(a, l, sLL);
            l2l_ready = true;
          }
          __syncthreads();
          l2l_quad_group(a, l, nl2l, b - nchu, sLL, wsm, warp, lane);
          continue;
        }
        const int pb = a.ch_beg[l][b], pe = a.ch_end[l][b];
        const int S = a.S[l], O = a.O[l];
        __syncthreads();                                      // sT of the previous chunk is done
        if (!(b0 == rb && pf_c == b && pf_cl == l)) stage_chunk(a, l, b, sT);
        __syncthreads();
        // two pairs per warp pass, sharing the operator rows read from shared memory
        for (int pi = pb + 2 * warp; pi < pe; pi += 2 * nw()) {
          const bool two = pi + 1 < pe;
          const int srcA = a.pr_src[l][pi], tgtA = a.pr_tgt[l][pi];
          const int srcB = two ? a.pr_src[l][pi + 1] : srcA, tgtB = two ? a.pr_tgt[l][pi + 1] : tgtA;
          const C phA = from_d<C>(phase_m(a.alpha, a.pr_img[l][pi]));
          const C phB = two ? from_d<C>(phase_m(a.alpha, a.pr_img[l][pi + 1])) : C{0, 0};
          __syncwarp();
          for (int m = lane; m < P; m += 32) {
            wsm[m] = phA * ldcg(a.M[l] + (size_t)srcA * S + O + m);
            wsm[P + m] = phB * ldcg(a.M[l] + (size_t)srcB * S + O + m);
          }
          __syncwarp();
          C* LA = a.L[l] + (size_t)tgtA * S + O;
          C* LB = a.L[l] + (size_t)tgtB * S + O;
          warp_rowmv2(sT, P, wsm, wsm + P, lane, [&](int n, C rA, C rB) {
            atomic_add(LA + n, rA);
            if (two) atomic_add(LB + n, rB);
          });
        }
      }
    }
    if (a.bdone && threadIdx.x == 0) a.bdone[(size_t)(ks - 1) * G + bid] = gtimer();
    // box-form L2L with the quadrant operators staged in shared memory, one
    // quadrant at a time (the FP64 product's hi and lo tables)
    const bool sl2l = ql2l || (!top && Pp * P <= TSIZE && P <= 64 && Pp <= PF_NCOEF);
    if (sl2l && !ql2l) l2l_staged(a, l, nl2l, wfirst, wstride, sT, wsm, lane, bid);
    const int nm2l = (wpair && !tcl) ? a.npair[l] : 0;
    const int jst = nbst + l - 1;
    const int r0 = a.near_first ? (jst == 0 ? 0 : NI) : (int)((int64_t)NI * jst / nst);
    const int r1 = a.near_first ? NI : (int)((int64_t)NI * (jst + 1) / nst);
    const int nitem = nl2l + nm2l + (r1 - r0);
    int4 nd;
    const int inear = first_near(a, wfirst, wstride, nl2l + nm2l, nitem, r0, &nd);
    for (int i = wfirst; i < nl2l + nm2l; i += wstride) {
      if (i < nl2l) {
        if (sl2l) continue;
        if (top && a.top3 && l == 1) {
          // the root's part of L(1) straight from the four level-1 multipoles
          // (those of empty level-1 boxes are kept at zero)
          const int bi = i / P, n = i - bi * P;
          const int box = a.ne[1][bi], S1 = a.S[1], O1 = a.O[1];
          const C* A = a.root1 + ((size_t)box * S1 + O1 + n) * 4 * S1;
          C acc{0, 0};
          for (int u = lane; u < 4 * P; u += 32) {
            const int q = u / P, v = q * S1 + O1 + (u - q * P);
            acc += A[v] * ldcg(a.M[1] + v);
          }
          acc = wsum(acc);
          if (lane == 0) atomic_add(a.L[1] + (size_t)box * S1 + O1 + n, acc);
        } else if (top) {
          const int bi = i / P, n = i - bi * P;
          const int box = a.ne[l][bi], par = box >> 2, q = box & 3;
          const int S = a.S[l], O = a.O[l], Sp = a.S[l - 1], Op = a.O[l - 1];
          const C* A = a.l2l[l - 1] + (size_t)(q * Sp + Op) * S + O + n;
          C acc{0, 0};
          for (int m = lane; m < Pp; m += 32)
            acc += A[(size_t)m * S] * ldcg(a.L[l - 1] + (size_t)par * Sp + Op + m);
          acc = wsum(acc);
          if (lane == 0) atomic_add(a.L[l] + (size_t)box * S + O + n, acc);
        } else {
          // the generic form, with the offsets of the used coefficients (see M2M)
          const int box = a.ne[l][i], par = box >> 2, q = box & 3;
          const int S = a.S[l], O = a.O[l], Sp = a.S[l - 1], Op = a.O[l - 1];
          __syncwarp();
          for (int m = lane; m < Pp; m += 32) wsm[m] = ldcg(a.L[l - 1] + (size_t)par * Sp + Op + m);
          __syncwarp();
          for (int n = lane; n < P; n += 32)
            atomic_add(a.L[l] + (size_t)box * S + O + n,
                       colmv(a.l2l[l - 1] + (size_t)(q * Sp + Op) * S + O + n, S, wsm, Pp));
        }
        continue;
      }
      const int pi = i - nl2l;
      const int src = a.pr_src[l][pi], tgt = a.pr_tgt[l][pi];
      const C phs = from_d<C>(phase_m(a.alpha, a.pr_img[l][pi]));
      if (a.m2ltl[l]) {
        // the FP64 product in double-float arithmetic on the FP32 pipes: the
        // phased source multipole split into hi and lo parts, the operator
        // read from its hi and lo tables
        cplxf* wh = reinterpret_cast<cplxf*>(wsm);
        cplxf* wl = wh + PF_NCOEF;
        __syncwarp();
        for (int m = lane; m < P; m += 32) {
          const cplx v = to_d(phs * ldcg(a.M[l] + (size_t)src * P + m));
          wh[m] = cplxf{(float)v.re, (float)v.im};
          wl[m] = split_lo(v);
        }
        __syncwarp();
        const size_t ob = (size_t)a.pr_off[l][pi] * P * P;
        const cplxf* Th = a.m2lth[l] + ob;
        const cplxf* Tl = a.m2ltl[l] + ob;
        for (int n = lane; n < P; n += 32) {
          dflt re{0, 0}, im{0, 0};
#pragma unroll 4
          for (int m = 0; m < P; ++m) dd_cmac(re, im, Th[(size_t)m * P + n], Tl[(size_t)m * P + n], wh[m], wl[m]);
          atomic_add(a.L[l] + (size_t)tgt * P + n, from_d<C>(cplx{dd_value(re), dd_value(im)}));
        }
        continue;
      }
      const int S = a.S[l], O = a.O[l];
      const C* To = a.m2lt[l] + (size_t)a.pr_off[l][pi] * S * S + (size_t)O * S + O;
      __syncwarp();
      for (int m = lane; m < P; m += 32) wsm[m] = phs * ldcg(a.M[l] + (size_t)src * S + O + m);
      __syncwarp();
      for (int n = lane; n < P; n += 32) atomic_add(a.L[l] + (size_t)tgt * S + O + n, colmv(To + n, S, wsm, P));
    }
    near_items(a, inear, nitem, wstride, r0, nl2l + nm2l, nd, lane);
    if (l < D) prefetch(ks, -1, l + 1);     // the next D stage's operators, staged ahead
    if (!group_barrier(a.bar, a.err, a.wait_ns, G, bid, a.arrive ? a.arrive + (size_t)(ks - 1) * G : nullptr)) {
      tc_leave();
      return false;
    }
    stage_stamp(a.stamp, ks++, bid);
  }

  // ------------------------------------------------------------ E: L2P + near field, combination of eq. 9
  // one lane per element (32 consecutive sorted elements per warp item): the
  // coefficients lie coefficient-major, so the lanes' loads are contiguous, and
  // no lane sums need a reduction
  {
    const int PD = a.P[D], SD = a.S[D], OD = a.O[D];
    const C c2 = from_d<C>(a.c2);
    const int nit = (a.E + 31) >> 5;
    for (int it = wfirst; it < nit; it += wstride) {
      const int s = (it << 5) + lane;
      if (s >= a.E) continue;
      const int box = a.ne[D][a.s_li[s]];
      const C* Lb = a.L[D] + (size_t)box * SD + OD;
      const C* cs = a.l2p + s + (size_t)OD * a.E;
      C uf{0, 0}, df{0, 0};
      if (a.l2pl && a.l2p_dd) {
        // FP64 product: L2P in double-float arithmetic from the caches' hi and lo parts
        const cplxf* ch = a.l2ph + s + (size_t)OD * a.E;
        const cplxf* cl = a.l2pl + s + (size_t)OD * a.E;
        dflt ur{0, 0}, ui{0, 0}, dr{0, 0}, di{0, 0};
#pragma unroll 8
        for (int t = 0; t < PD; ++t) {
          const cplx Lt = to_d(ldcg(Lb + t));
          const cplxf Lh{(float)Lt.re, (float)Lt.im}, Ll = split_lo(Lt);
          dd_cmac(ur, ui, ch[(size_t)t * a.E], cl[(size_t)t * a.E], Lh, Ll);
          dd_cmac(dr, di, ch[(size_t)(SD + t) * a.E], cl[(size_t)(SD + t) * a.E], Lh, Ll);
        }
        uf = from_d<C>(cplx{dd_value(ur), dd_value(ui)});
        df = from_d<C>(cplx{dd_value(dr), dd_value(di)});
      } else {
#pragma unroll 16
        for (int t = 0; t < PD; ++t) {
          const C Lt = ldcg(Lb + t);
          uf += cs[(size_t)t * a.E] * Lt;
          df += cs[(size_t)(SD + t) * a.E] * Lt;
        }
      }
      // back to the element's true position: times alpha^{m0} = conj(alpha^{-m0})
      const int e = a.perm[s];
      if (a.rsum) {
        // FP32 product with near sums in differences: add the row-sum part R_s psi_s
        // and combine in FP64
        const cplx p0 = a.ph[s] * a.x[2 * e], p1 = a.ph[s] * a.x[2 * e + 1];
        const cplx* R = a.rsum + 4 * (size_t)s;
        const cplx u = to_d(uf + ldcg(a.Un + 2 * s)) + R[0] * p0 + R[1] * p1;
        const cplx du = to_d(df + ldcg(a.Un + 2 * s + 1)) + R[2] * p0 + R[3] * p1;
        const cplx po = conj(a.ph[s]);
        a.y[2 * e] = ldcg(a.y + 2 * e) + po * u;
        a.y[2 * e + 1] = ldcg(a.y + 2 * e + 1) + a.c2 * (po * du);
        continue;
      }
      const C po = from_d<C>(conj(a.ph[s]));
      const C u = po * (uf + ldcg(a.Un + 2 * s));
      const C du = c2 * (po * (df + ldcg(a.Un + 2 * s + 1)));
      a.y[2 * e] = ldcg(a.y + 2 * e) + to_d(u);
      a.y[2 * e + 1] = ldcg(a.y + 2 * e + 1) + to_d(du);
    }
  }
  __syncthreads();
  stage_stamp(a.stamp, ks++, bid);
  tc_leave();
  return true;
}

// The single-launch product over the whole grid (a cooperative launch).
template <class C, bool TC>
__global__ void __launch_bounds__(TC ? 2 * FB : FB, TC ? 1 : (sizeof(C) == sizeof(cplx) ? 3 : 2))
    matvec_fused_kernel(const __grid_constant__ FusedArgs<C> a) {
  // a GMRES cycle that has already converged skips the products queued after it
  if (a.done && *(volatile const int*)a.done != 0) return;
  fused_body<C, TC>(a, (int)blockIdx.x, (int)gridDim.x);
}

// Threads per block of a form of the single-launch product.
constexpr int fused_threads(bool tc) { return tc ? 2 * FB : FB; }

template <class C>
size_t fused_smem(int maxfiber, int treg, size_t tcb, int nwarp) {
  const size_t a = (size_t)treg + (size_t)nwarp * PF_NCOEF; // stages B, D
  const size_t f = 2 * (size_t)maxfiber + 512;              // fiber part of stage A, with its twiddles (FP64 FFTs)
  return std::max({sizeof(C) * a, sizeof(cplx) * f, tcb});  // tcb: tensor-core M2L operands
}

// After a bounded device-side wait gave up, the barrier words and the error
// flag are in an unknown state: clear them (on the handle's stream) before the
// next launch that uses them.
cudaError_t reset_device_waits(pfmbem* h) {
  if (!h->fz_dirty) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (h->fz_bar) e = cudaMemsetAsync(h->fz_bar, 0, 2 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess && h->arn_bar) e = cudaMemsetAsync(h->arn_bar, 0, 2 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess && h->fz_err) e = cudaMemsetAsync(h->fz_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) h->fz_dirty = false;
  return e;
}

// Operators, vectors and work lists of one product of the single-launch kernel.
// Coefficients per expansion at level l in the single-launch product.  The
// FP32 product may run at a lower order than the FP64 one (the central
// sub-blocks of the same tables); only with the folded top of the tree (level 3
// present), whose paths all take the strides.
int fused_P(const pfmbem* h, int l, bool f32) {
  const Level& L = h->lev[l];
  const bool reduce = f32 && h->m2m31 != nullptr && h->D >= 3;
  const int pu = reduce ? std::min(L.p, std::max(1, L.p32)) : L.p;
  return 2 * pu + 1;
}

template <class C>
cudaError_t fill_args(pfmbem* h, const cplx* x, cplx* y, const int* done, FusedArgs<C>& a) {
  a = FusedArgs<C>{};
  a.done = done;
  a.tws_off = 2 * h->max_fiber;
  a.treg = sizeof(C) == sizeof(cplxf) ? std::max(TSIZE, h->fz_treg32) : TSIZE;
  a.tregL = sizeof(C) == sizeof(cplxf) && h->fz_tcb32 == 0 ? h->fz_tregL32 : 0;
  a.nr_meta = reinterpret_cast<const longlong2*>(h->nr_meta);
  static const bool rows = std::getenv("PFMBEM_NEAR_ROWS") != nullptr;   // measurement: whole rows
  a.nr_piece = h->nr_piece;
  a.npiece = (sizeof(C) == sizeof(cplxf) && h->fz_dlo && h->nr_piece && !rows) ? h->nr_npiece : 0;
  a.tc_any = 0;
  for (int l = 0; l <= h->D; ++l) {
    const Level& L = h->lev[l];
    const int kp = tc::kpad(fused_P(h, l, sizeof(C) == sizeof(cplxf)));
    const bool on = sizeof(C) == sizeof(cplxf) && l >= 1 && h->fz_tcb32 > 0 && L.tc_fused && L.tc_Bf &&
                    L.tc_ntile > 0 && kp <= TC_KPMAX;
    a.tc_kp[l] = on ? kp : 0;
    a.tc_ntile[l] = on ? L.tc_ntile : 0;
    // offset groups per tile: about two block items per block of the grid
    // (PFMBEM_TC_GROUPS overrides, for measurement)
    static const char* tg = std::getenv("PFMBEM_TC_GROUPS");
    const int G = h->fz_grid32 > 0 ? h->fz_grid32 : 1;
    a.tc_ngrp[l] = on ? std::max(1, std::min(49, (2 * G + L.tc_ntile - 1) / L.tc_ntile)) : 1;
    if (on && tg) a.tc_ngrp[l] = std::max(1, std::min(49, std::atoi(tg)));
    a.tc_box[l] = L.tc_box;
    a.tc_noff[l] = L.tc_noff;
    a.tc_offs[l] = L.tc_offs;
    a.tc_src[l] = L.tc_src;
    a.tc_img[l] = L.tc_img;
    a.tc_B[l] = L.tc_Bf;
    a.tc_any |= on ? 1 : 0;
  }
  a.E = h->E;
  a.D = h->D;
  a.nroot = h->nroot;
  a.perm = h->s_perm;
  a.ph = h->s_ph;
  a.opos = h->o_pos;
  a.x = x;
  a.y = y;
  for (int l = 0; l <= h->D; ++l) {
    const Level& L = h->lev[l];
    a.nne[l] = L.nne;
    const int pu = (fused_P(h, l, sizeof(C) == sizeof(cplxf)) - 1) / 2;
    a.P[l] = 2 * pu + 1;
    a.S[l] = L.P;
    a.O[l] = L.p - pu;
    a.ne[l] = L.ne;
    a.bb[l] = L.box_begin;
    a.be[l] = L.box_end;
    a.nbox[l] = L.nbox;
    a.nch[l] = L.nchunk;
    a.ch_off[l] = L.ch_off;
    a.ch_beg[l] = L.ch_beg;
    a.ch_end[l] = L.ch_end;
    a.pr_tgt[l] = L.pr_tgt;
    a.pr_src[l] = L.pr_src;
    a.pr_img[l] = L.pr_img;
    a.pr_off[l] = L.pr_off;
    a.npair[l] = (int)L.nil;
    if constexpr (sizeof(C) == sizeof(cplxf)) {
      a.m2m[l] = L.m2mf; a.l2l[l] = L.l2lf; a.m2lt[l] = L.m2ltf; a.M[l] = L.Mf; a.L[l] = L.Lf;
    } else {
      a.m2m[l] = L.m2m; a.l2l[l] = L.l2l; a.m2lt[l] = L.m2lt; a.M[l] = L.M; a.L[l] = L.L;
    }
  }
  a.s_li = h->s_li;
  if constexpr (sizeof(C) == sizeof(cplxf)) {
    a.Un = h->Unf;
    a.dens = h->densf; a.root = h->rootf; a.rootc = h->rootcf; a.p2m = h->p2m_cf; a.l2p = h->l2p_cf;
    // near sums in differences and FP64 same-fiber FFTs (PFMBEM_FP32_PLAIN=1 turns
    // both off, for measurement)
    static const bool plain = std::getenv("PFMBEM_FP32_PLAIN") != nullptr;
    if (!plain && h->fz_dlo && h->fz_rsum) {
      a.dlo = h->fz_dlo;
      a.rsum = h->fz_rsum;
    }
    if (!plain && h->fh_val) {
      a.fh64 = h->fh_val;
      a.tw64 = h->tw;
    }
    if (!plain && h->fz_frs) a.frs = h->fz_frs;
    a.m2m31 = h->m2m31f; a.root1 = h->root1f;
    a.nc_val = h->nc_valf; a.fb_val = h->fb_valf; a.fh_val = h->fh_valf; a.tw = h->twf;
  } else {
    a.Un = h->Un;
    a.dens = h->dens; a.root = h->root; a.rootc = h->rootc; a.p2m = h->p2m_c; a.l2p = h->l2p_c;
    // (PFMBEM_NEAR_FP64 selects FP64 near sums and M2L instead, for measurement)
    static const bool near64 = std::getenv("PFMBEM_NEAR_FP64") != nullptr;
    if (near64 || !h->dens_dd) {
      cudaError_t e = k_near64(h);                  // FP64 blocks, formed on first use
      if (e != cudaSuccess) return e;
    }
    if (h->nc_vall && h->dens_dd && !near64) {
      a.nc_lo = h->nc_vall;
      a.nc_hi = h->nc_valf;
      a.dens_dd = h->dens_dd;
      for (int l = 1; l <= h->D; ++l) {
        a.m2lth[l] = h->lev[l].m2ltf;
        a.m2ltl[l] = h->lev[l].m2ltl;
      }
      for (int l = 0; l < h->D; ++l) {
        a.m2mh[l] = h->lev[l].m2mf;
        a.m2ml[l] = h->lev[l].m2ml;
        if (h->lev[l].l2ll) {
          a.l2lh[l] = h->lev[l].l2lf;
          a.l2ll[l] = h->lev[l].l2ll;
        }
      }
      a.p2mh = h->p2m_cf;
      a.p2ml = h->p2m_cl;
      if (h->l2p_cl) {
        a.l2ph = h->l2p_cf;
        a.l2pl = h->l2p_cl;
        static const bool l2pdd = std::getenv("PFMBEM_L2P_DD") != nullptr;
        a.l2p_dd = l2pdd ? 1 : 0;
      }
    }
    a.m2m31 = h->m2m31; a.root1 = h->root1;
    a.nc_val = h->nc_val; a.fb_val = h->fb_val; a.fh_val = h->fh_val; a.tw = h->tw;
  }
  a.nc_base = h->nc_base;
  a.nc_sbase = h->nc_sbase;
  a.nc_src = h->nc_src;
  a.nchunk = h->fz_nchunk;
  a.fb_chunk = h->fz_chunk;
  a.nfft = h->fz_nfft;
  a.fft_fib = h->fz_fft;
  a.fh_base = h->fh_base;
  a.foff = h->fib_off;
  a.fb_base = h->fb_base;
  a.circ = h->fb_circ;
  a.alpha = h->alpha;
  a.c2 = cplx{h->c2re, h->c2im};
  a.bar = h->fz_bar + (sizeof(C) == sizeof(cplxf) ? 1 : 0);   // one counter per grid size
  a.err = h->fz_err;
  a.wait_ns = h->opt.wait_us > 0 ? 1000ull * (unsigned long long)h->opt.wait_us : 1000000000ull;
  return cudaSuccess;
}

template <class C>
cudaError_t launch_fused(pfmbem* h, const cplx* x, cplx* y, bool f32, const int* done) {
  FusedArgs<C> a;
  {
    cudaError_t e = reset_device_waits(h);
    if (e == cudaSuccess) e = fill_args<C>(h, x, y, done, a);
    if (e != cudaSuccess) return e;
  }
  static const bool stamps = std::getenv("PFMBEM_STAGE_TIMES") != nullptr;
  a.stamp = stamps ? h->fz_stamp : nullptr;
  // diagnostic (PFMBEM_BLOCK_TIMES set, with PFMBEM_STAGE_TIMES): every block's
  // arrival at every barrier
  static const bool btimes = std::getenv("PFMBEM_BLOCK_TIMES") != nullptr;
  a.arrive = stamps && btimes ? h->fz_arrive : nullptr;
  a.bdone = a.arrive ? h->fz_arrive + (size_t)16 * 1024 : nullptr;
  const int grid = f32 ? h->fz_grid32 : h->fz_grid64;
  // the tensor-core form: FP32 product with tensor-core M2L levels
  const bool tc = f32 && h->fz_tcb32 > 0;
  const int nthr = fused_threads(tc), nwarp = nthr / 32;
  // several roots: L(0) takes one warp per root coefficient (its only form)
  if (h->nroot > 1 && (int64_t)h->lev[0].nne * h->lev[0].P > (int64_t)grid * nwarp) return cudaErrorInvalidConfiguration;
  // the fiber part's blocks in stage A, in proportion to its block items
  // against the P2M warp items (one leaf per warp)
  {
    const int nf = h->fz_nfft + h->fz_nchunk;
    const double wa = (double)h->lev[h->D].nne / nwarp;
    const int fb = (int)((double)grid * nf / (nf + wa) + 0.5);
    a.fblk = grid >= 16 ? std::max(1, std::min({fb, nf, grid - grid / 4})) : 0;
  }
  // M2L: warp per pair in FP64, whose per-pair cost the FP64 pipe sets; staged
  // chunks in FP32 (PFMBEM_M2L_WARP=0/1 overrides, for measurement)
  static const char* mw = std::getenv("PFMBEM_M2L_WARP");
  a.m2l_warp = mw ? std::atoi(mw) != 0 : !f32;
  static const bool nf = std::getenv("PFMBEM_NEAR_FIRST") != nullptr;
  a.near_first = nf ? 1 : 0;
  // levels 1 and 0 inside the level-2 stage when the tree has level 3 and the
  // three levels' coefficients fit one item per warp
  {
    const int64_t w = (int64_t)grid * nwarp;
    a.top3 = h->m2m31 != nullptr &&
             (int64_t)h->lev[2].nne * h->lev[2].P + (int64_t)h->lev[1].nne * h->lev[1].P + 4 * h->lev[0].P <= w;
  }
  const size_t smem = fused_smem<C>(h->max_fiber, a.treg + a.tregL, tc ? h->fz_tcb32 : 0, nwarp);
  const void* fn = tc ? (const void*)matvec_fused_kernel<cplxf, true> : (const void*)matvec_fused_kernel<C, false>;
  {
    // the kernel's dynamic shared-memory limit is process-wide: raise it to
    // this launch's need (another handle may have set a smaller one)
    static std::atomic<size_t> set_max[2]{{0}, {0}};
    std::atomic<size_t>& sm = set_max[tc ? 1 : 0];
    size_t cur = sm.load();
    if (smem > cur) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      while (smem > cur && !sm.compare_exchange_weak(cur, smem)) {
      }
    }
  }
  void* args[] = {&a};
  const int ph = PH_FUSED + (f32 ? 16 : 0);
  prof_begin(h, ph);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(nthr), args, smem, h->stream);
  prof_end(h, ph);
  if (e == cudaSuccess && a.stamp) {
    // diagnostic (PFMBEM_STAGE_TIMES set): stage durations of this launch on stderr
    unsigned long long t[32];
    e = cudaMemcpyAsync(t, a.stamp, sizeof(t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) {
      const int n = 2 * h->D + 3 - (a.top3 ? 2 : 0);
      std::fprintf(stderr, "pfmbem fused %s grid %d smem %zu stages (us):", f32 ? "f32" : "f64", grid, smem);
      for (int i = 1; i < n; ++i) std::fprintf(stderr, " %.1f", 1e-3 * (double)(t[i] - t[i - 1]));
      std::fprintf(stderr, "  total %.1f\n", 1e-3 * (double)(t[n - 1] - t[0]));
      if (a.arrive && grid <= 1024) {
        // per stage: the blocks' arrivals at its closing barrier after the
        // stage's start (block 0 leaving the previous barrier): min, median,
        // 90th percentile, max (us) and the last block
        std::vector<unsigned long long> arr((size_t)(n - 1) * grid), bd((size_t)3 * 8192, 0);
        e = cudaMemcpy(arr.data(), a.arrive, sizeof(unsigned long long) * arr.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
          e = cudaMemcpy(bd.data(), a.bdone, sizeof(unsigned long long) * bd.size(), cudaMemcpyDeviceToHost);
        for (int i = 1; e == cudaSuccess && i < n - 1; ++i) {
          std::vector<double> d(grid), q;
          int last = 0;
          for (int b = 0; b < grid; ++b) {
            d[b] = 1e-3 * ((double)arr[(size_t)(i - 1) * grid + b] - (double)t[i - 1]);
            if (d[b] > d[last]) last = b;
            const unsigned long long x = bd[(size_t)(i - 1) * grid + b];
            if (x > t[i - 1] && x < t[i]) q.push_back(1e-3 * ((double)x - (double)t[i - 1]));
          }
          std::vector<double> srt = d;
          std::sort(srt.begin(), srt.end());
          std::sort(q.begin(), q.end());
          // block 'last''s own marks: operators staged, children gathered (M2M), block items done
          auto mark = [&](size_t slot) {
            const unsigned long long x = bd[slot + (size_t)(i - 1) * grid + last];
            return x > t[i - 1] && x < t[i] ? 1e-3 * ((double)x - (double)t[i - 1]) : -1.0;
          };
          std::fprintf(stderr,
                       "pfmbem fused %s stage %d arrivals (us): %.1f %.1f %.1f %.1f last block %d, stage %.1f; "
                       "block items done: median %.1f max %.1f; last block: staged %.1f gathered %.1f items %.1f\n",
                       f32 ? "f32" : "f64", i, srt[0], srt[grid / 2], srt[(9 * grid) / 10], srt[grid - 1], last,
                       1e-3 * (double)(t[i] - t[i - 1]), q.empty() ? 0.0 : q[q.size() / 2],
                       q.empty() ? 0.0 : q.back(), mark(8192), mark(16384), mark(0));
        }
        cudaMemsetAsync(a.bdone, 0, sizeof(unsigned long long) * bd.size(), h->stream);
      }
    }
  }
  return e;
}

template <class C, bool TC>
int fused_grid(int maxfiber, int treg, size_t tcb) {
  const void* fn = (const void*)matvec_fused_kernel<C, TC>;
  const int nthr = fused_threads(TC);
  const size_t smem = fused_smem<C>(maxfiber, treg, tcb, nthr / 32);
  // the limit only grows: handles made earlier keep theirs
  int cur = 0;
  {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) cur = fa.maxDynamicSharedSizeBytes;
    cudaGetLastError();
  }
  if ((int)smem > cur && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, nsm = 0, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nthr, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // resident blocks per SM: three for the FP64 product, whose stages are bound
  // by the FP64 pipes of all sub-partitions; two for the FP32 product, whose
  // stages are short and pay less for a barrier over fewer blocks; one of 512
  // threads in the tensor-core form (PFMBEM_FUSED_BLOCKS_PER_SM overrides the
  // first two, for measurement)
  static const char* bps = std::getenv("PFMBEM_FUSED_BLOCKS_PER_SM");
  const int cap = TC ? 1 : bps ? std::max(1, std::atoi(bps)) : (sizeof(C) == sizeof(cplx) ? 3 : 2);
  return nsm * std::min(per, cap);
}


}  // namespace

// Row sums R_s = sum_j B_sj of the cached near blocks (hi + lo, in FP64) for the
// FP32 product's near sums in differences: one warp per sorted element.
__global__ void near_rowsum_kernel(int E, int D, const int* __restrict__ s_li, const int* __restrict__ ne,
                                   const int* __restrict__ bb, const int* __restrict__ nc_sbase,
                                   const int64_t* __restrict__ nc_base, const cplxf* __restrict__ hi,
                                   const cplxf* __restrict__ lo, cplx* __restrict__ rsum) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= E) return;
  const int li = s_li[s];
  const int t = s - bb[ne[li]];
  const int ns = nc_sbase[li + 1] - nc_sbase[li];
  const int64_t r = nc_base[li] + (int64_t)t * ns * 4;
  // double-float sums (about 48 bits) on the FP32 pipes; FP64 adds would run at
  // 1/64 of their rate
  dflt ar[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}}, ai[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int j = lane; j < ns; j += 32)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const cplxf h = hi[r + 4 * j + q], l = lo[r + 4 * j + q];
      ar[q] = dd_add(ar[q], dflt{h.re, l.re});
      ai[q] = dd_add(ai[q], dflt{h.im, l.im});
    }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const dflt vr = dd_wsum(ar[q]), vi = dd_wsum(ai[q]);
    if (lane == 0) rsum[4 * (size_t)s + q] = cplx{dd_value(vr), dd_value(vi)};
  }
}

// Row sums of the same-fiber rows split by column parity: frs[row][q] = sum over
// the columns c = q mod 2 of the FP64 row (a circulant fiber's rows are
// rotations of its first row pair by whole elements, so they share its sums).
// One warp per row of a fiber applied by rows.
__global__ void fiber_rowsum_kernel(int nrow, const int* __restrict__ row_fiber, const int* __restrict__ foff,
                                    const int64_t* __restrict__ fb_base, const int* __restrict__ circ,
                                    const cplx* __restrict__ fb_val, cplx* __restrict__ frs) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= nrow) return;
  const int fb = row_fiber[2 * i], r = row_fiber[2 * i + 1];
  const int f0 = foff[fb], n2 = 2 * (foff[fb + 1] - f0);
  const cplx* row = fb_val + fb_base[fb] + (int64_t)(circ[fb] ? (r & 1) : r) * n2;
  cplx e{0, 0}, o{0, 0};
  for (int c = lane; c < n2; c += 32) {
    if (c & 1) o += row[c];
    else e += row[c];
  }
  e = wsum(e);
  o = wsum(o);
  if (lane == 0) {
    frs[2 * (size_t)(2 * f0 + r)] = e;
    frs[2 * (size_t)(2 * f0 + r) + 1] = o;
  }
}

// Device tables of the single-launch product that read uploaded lists (buffers
// allocated by the caller): the near blocks' row sums.
cudaError_t k_fused_tables(pfmbem* h) {
  const int D = h->D;
  if (h->fz_frs && h->fz_nrowsum > 0)
    fiber_rowsum_kernel<<<(h->fz_nrowsum * 32 + 255) / 256, 256, 0, h->stream>>>(
        h->fz_nrowsum, h->fz_rowfib, h->fib_off, h->fb_base, h->fb_circ, h->fb_val, h->fz_frs);
  const Level& Lf = h->lev[D];
  if (h->fz_rsum)
    near_rowsum_kernel<<<(h->E * 32 + 255) / 256, 256, 0, h->stream>>>(h->E, D, h->s_li, Lf.ne, Lf.box_begin,
                                                                      h->nc_sbase, h->nc_base, h->nc_valf,
                                                                      h->nc_vall, h->fz_rsum);
  return cudaGetLastError();
}

// ------------------------------------------------ triangle tree: double-float M2L
// hi and lo FP32 parts of n FP64 values: out[i] = hi, out[n + i] = lo.
__global__ void split_hl_kernel(size_t n, const cplx* __restrict__ a, cplxf* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    out[i] = cplxf{(float)a[i].re, (float)a[i].im};
    out[n + i] = split_lo(a[i]);
  }
}

// M2L of the triangle tree's offset groups (chunks of at most 16 pairs of one
// offset) in double-float arithmetic: the FP64 result on the FP32 pipes, which
// GB300 issues at 64 times its FP64 rate.  One block per chunk stages the
// offset's operator as hi and lo parts ([P][P+1] each, padded rows); a warp per
// pair splits its phased source multipole alpha^m M(src) into hi and lo, sums
// each target coefficient with error-free products and sums (about 48 bits)
// and adds it to L(tgt) in FP64.  L(tgt) holds the L2L part already.
__global__ void tri_m2l_dd_kernel(int P, int noff, const int* __restrict__ chunk_off, const int* __restrict__ chunk_beg,
                                  const int* __restrict__ chunk_end, const int* __restrict__ ptgt,
                                  const int* __restrict__ psrc, const int* __restrict__ pimg,
                                  const cplxf* __restrict__ Thl, const cplx* __restrict__ M, cplx alpha,
                                  cplx* __restrict__ L) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplxf* sh = reinterpret_cast<cplxf*>(smraw);          // [P][P+1] hi
  cplxf* sl = sh + (size_t)P * (P + 1);                  // [P][P+1] lo
  cplxf* sm = sl + (size_t)P * (P + 1);                  // [warps][2][P] source hi, lo
  const int o = chunk_off[blockIdx.x];
  const int pb = chunk_beg[blockIdx.x], pe = chunk_end[blockIdx.x];
  const size_t PP = (size_t)P * P;
  const cplxf* Th = Thl + (size_t)o * PP;
  const cplxf* Tl = Thl + (size_t)noff * PP + (size_t)o * PP;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    const int r = i / P, c = i - r * P;
    sh[r * (P + 1) + c] = Th[i];
    sl[r * (P + 1) + c] = Tl[i];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  cplxf* wh = sm + (size_t)warp * 2 * P;
  cplxf* wl = wh + P;
  __syncthreads();
  for (int pi = pb + warp; pi < pe; pi += nw) {
    const int src = psrc[pi], tgt = ptgt[pi];
    const cplx ph = phase_m(alpha, pimg[pi]);
    __syncwarp();
    for (int n = lane; n < P; n += 32) {
      const cplx v = ph * M[(size_t)src * P + n];
      wh[n] = cplxf{(float)v.re, (float)v.im};
      wl[n] = split_lo(v);
    }
    __syncwarp();
    for (int l = lane; l < P; l += 32) {
      const cplxf* rh = sh + (size_t)l * (P + 1);
      const cplxf* rl = sl + (size_t)l * (P + 1);
      dflt re{0, 0}, im{0, 0};
      for (int n = 0; n < P; ++n) dd_cmac(re, im, rh[n], rl[n], wh[n], wl[n]);
      atomic_add(L + (size_t)tgt * P + l, cplx{dd_value(re), dd_value(im)});
    }
  }
}

// M2M and L2L of the triangle tree in double-float arithmetic, one block per
// box and a thread per output coefficient; the operators' hi parts first, then
// their lo parts (nop operators of [Pc][P] for M2M, [Pp][P] for L2L, rows of the
// input coefficient, as the FP64 tables).  M2M: M(box) = sum over the non-empty
// children ch (nch per box) of A_aidx[ch] M(ch).
__global__ void tri_m2m_dd_kernel(const int* __restrict__ ne, int P, int Pc, int nop, const cplxf* __restrict__ Ahl,
                                  const int* __restrict__ cbb, const int* __restrict__ cbe,
                                  const cplx* __restrict__ Mc, cplx* __restrict__ Mp, int nch,
                                  const int* __restrict__ aidx) {
  const int box = ne[blockIdx.x];
  __shared__ cplxf sh[PF_NCOEF], sl[PF_NCOEF];
  const size_t lo = (size_t)nop * Pc * P;
  dflt re{0, 0}, im{0, 0};
  for (int q = 0; q < nch; ++q) {
    const int ch = nch * box + q;
    if (cbb[ch] >= cbe[ch]) continue;   // empty child (uniform across the block)
    __syncthreads();
    for (int i = threadIdx.x; i < Pc; i += blockDim.x) {
      const cplx v = Mc[(size_t)ch * Pc + i];
      sh[i] = cplxf{(float)v.re, (float)v.im};
      sl[i] = split_lo(v);
    }
    __syncthreads();
    if (threadIdx.x < P) {
      const cplxf* ah = Ahl + (size_t)aidx[ch] * Pc * P + threadIdx.x;
      for (int m = 0; m < Pc; ++m) dd_cmac(re, im, ah[(size_t)m * P], ah[lo + (size_t)m * P], sh[m], sl[m]);
    }
  }
  if (threadIdx.x < P) Mp[(size_t)box * P + threadIdx.x] = cplx{dd_value(re), dd_value(im)};
}

// L2L: L(box) = B_pidx[box] L(parent), the parent box / nchp.
__global__ void tri_l2l_dd_kernel(const int* __restrict__ ne, int P, int Pp, int nop, const cplxf* __restrict__ Bhl,
                                  const cplx* __restrict__ Lp, cplx* __restrict__ L, int nchp,
                                  const int* __restrict__ pidx) {
  const int box = ne[blockIdx.x];
  __shared__ cplxf sh[PF_NCOEF], sl[PF_NCOEF];
  const int par = box / nchp;
  for (int i = threadIdx.x; i < Pp; i += blockDim.x) {
    const cplx v = Lp[(size_t)par * Pp + i];
    sh[i] = cplxf{(float)v.re, (float)v.im};
    sl[i] = split_lo(v);
  }
  __syncthreads();
  if (threadIdx.x < P) {
    const size_t lo = (size_t)nop * Pp * P;
    const cplxf* bh = Bhl + (size_t)pidx[box] * Pp * P + threadIdx.x;
    dflt re{0, 0}, im{0, 0};
    for (int m = 0; m < Pp; ++m) dd_cmac(re, im, bh[(size_t)m * P], bh[lo + (size_t)m * P], sh[m], sl[m]);
    L[(size_t)box * P + threadIdx.x] = cplx{dd_value(re), dd_value(im)};
  }
}

cudaError_t k_tri_m2m_dd(pfmbem* h, int l) {
  const Level& a = h->lev[l];
  const Level& c = h->lev[l + 1];
  tri_m2m_dd_kernel<<<a.nne, ((a.P + 31) / 32) * 32, 0, h->stream>>>(a.ne, a.P, c.P, a.tri_nop, a.tri_m2m_hl,
                                                                     c.box_begin, c.box_end, c.M, a.M,
                                                                     l == 0 ? 6 : 4, c.pidx);
  return cudaGetLastError();
}

cudaError_t k_tri_l2l_dd(pfmbem* h, int l) {
  const Level& a = h->lev[l];
  const Level& pa = h->lev[l - 1];
  tri_l2l_dd_kernel<<<a.nne, ((a.P + 31) / 32) * 32, 0, h->stream>>>(a.ne, a.P, pa.P, pa.tri_nop, pa.tri_l2l_hl,
                                                                     pa.L, a.L, l == 1 ? 6 : 4, a.pidx);
  return cudaGetLastError();
}

// Level l's hi and lo operator parts from its FP64 M2L table.
// (and its M2M/L2L tables' parts, when the level has children)
cudaError_t k_tri_m2l_split(pfmbem* h, int l) {
  const Level& L = h->lev[l];
  const size_t n = (size_t)L.tri_noff * L.P * L.P;
  if (n > 0 && L.tri_m2l_hl)
    split_hl_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, h->stream>>>(n, L.m2l,
                                                                                               L.tri_m2l_hl);
  if (l < h->D && L.tri_m2m_hl && L.tri_l2l_hl) {
    const size_t ns = (size_t)L.tri_nop * L.P * h->lev[l + 1].P;
    split_hl_kernel<<<(unsigned)std::min<size_t>((ns + 255) / 256, 4096), 256, 0, h->stream>>>(ns, L.m2m,
                                                                                                L.tri_m2m_hl);
    split_hl_kernel<<<(unsigned)std::min<size_t>((ns + 255) / 256, 4096), 256, 0, h->stream>>>(ns, L.l2l,
                                                                                                L.tri_l2l_hl);
  }
  return cudaGetLastError();
}

// Level l's M2L by offset groups in double-float arithmetic (after its L2L).
cudaError_t k_tri_m2l_dd(pfmbem* h, int l) {
  const Level& L = h->lev[l];
  if (L.nchunk == 0) return cudaSuccess;
  const int nwarp = 8;
  const size_t smem = sizeof(cplxf) * (2 * (size_t)L.P * (L.P + 1) + 2 * (size_t)nwarp * L.P);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tri_m2l_dd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  tri_m2l_dd_kernel<<<L.nchunk, 32 * nwarp, smem, h->stream>>>(L.P, L.tri_noff, L.ch_off, L.ch_beg, L.ch_end,
                                                                L.pr_tgt, L.pr_src, L.pr_img, L.tri_m2l_hl, L.M,
                                                                h->alpha, L.L);
  return cudaGetLastError();
}

namespace {
}  // namespace

// The top operators of the fused product on stream st: R T_0 (root fold) and,
// with level 3 present, T_1 T_2 and R T_0 T_1 T_2; st must be ordered after the
// root operator and the M2M tables.
cudaError_t k_top_operators(pfmbem* h, cudaStream_t st) {
  const int P0 = h->lev[0].P, K = 4 * h->lev[1].P, nr = h->nroot;
  root_fold_kernel<<<(nr * nr * P0 * K + 7) / 8, 256, 0, st>>>(P0, K, nr, h->root, h->lev[0].m2m, h->rootc,
                                                                h->rootcf);
  // the multipoles of empty boxes are never written: keep them zero (the M2M
  // stages and M(1) read all four children without occupancy tests)
  for (int l = 1; l <= h->D; ++l) {
    const size_t nz = (size_t)h->lev[l].nbox * h->lev[l].P;
    cudaError_t e = cudaMemsetAsync(h->lev[l].M, 0, nz * sizeof(cplx), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->lev[l].Mf, 0, nz * sizeof(cplxf), st);
    if (e != cudaSuccess) return e;
  }
  if (h->m2m31) {
    const int P1 = h->lev[1].P, P2 = h->lev[2].P, P3 = h->lev[3].P;
    m2m31_kernel<<<(16 * P3 * P1 + 255) / 256, 256, 0, st>>>(P1, P2, P3, h->lev[1].m2m, h->lev[2].m2m, h->m2m31,
                                                             h->m2m31f);
    root1_kernel<<<(16 * P1 * P1 + 255) / 256, 256, 0, st>>>(P0, P1, h->lev[0].l2l, h->rootc, h->root1, h->root1f);
  }
  return cudaGetLastError();
}

// Prepares the fused path of a handle (grid sizes, barrier words); returns
// false when the device cannot run it, in which case the per-stage path is used.
cudaError_t k_fused_prepare(pfmbem* h, bool* ok) {
  *ok = false;
  // blocks with work in some stage: warps over boxes (A, B, D), blocks over
  // leaves and over fibers or fiber row chunks (fiber part of A)
  int need = std::max(h->lev[h->D].nne, h->fz_nchunk + h->fz_nfft);
  for (int l = 0; l <= h->D; ++l) need = std::max(need, (h->lev[l].nne + FW - 1) / FW);
  need = std::max(need, 1);
  // staging region of the FP32 product: room for the four stacked quadrant
  // operators of M2M and L2L at the FP32 orders, within about 100 KB per block
  // (two resident blocks per SM)
  {
    // only the levels that run box items (the others take one warp per
    // coefficient: more warps than boxes x coefficients, for two blocks per SM)
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t wst = (int64_t)2 * nsm * FW;
    int needm = 0, needl = 0;
    for (int l = 1; l <= h->D; ++l) {
      const int P = fused_P(h, l, true), Pp = fused_P(h, l - 1, true);
      if ((int64_t)h->lev[l].nne * P <= wst) continue;
      if (l < h->D && 4 * fused_P(h, l + 1, true) <= PF_NCOEF) needm = std::max(needm, 4 * fused_P(h, l + 1, true) * P);
      if (l >= 2 && Pp <= PF_NCOEF) needl = std::max(needl, 4 * Pp * P);
    }
    const int cap = (int)(100 * 1024 / sizeof(cplxf)) - 2 * FW * PF_NCOEF;   // room for 16 warps' scratch
    static const bool noquad = std::getenv("PFMBEM_NO_QUAD") != nullptr;   // measurement: per-quadrant staging
    h->fz_treg32 = noquad ? TSIZE : std::max(TSIZE, std::min(std::max(needm, needl), cap));
    // the plain form also keeps the L2L stack in a region of its own (staged
    // ahead beside the first M2L chunk's operator), within about 112 KB per block
    const int capL = (int)(112 * 1024 / sizeof(cplxf)) - FW * PF_NCOEF - h->fz_treg32;
    h->fz_tregL32 = !noquad && needl > 0 && needl <= capL ? needl : 0;
  }
  // tensor-core M2L levels of the FP32 product (their operands need up to
  // tc_smem_bytes(TC_KPMAX) of shared memory)
  h->fz_tcb32 = 0;
  for (int l = 1; l <= h->D; ++l) {
    const Level& L = h->lev[l];
    if (L.tc_fused && L.tc_Bf && L.tc_ntile > 0 && tc::kpad(fused_P(h, l, true)) <= TC_KPMAX)
      h->fz_tcb32 = std::max(h->fz_tcb32, tc_smem_bytes(tc::kpad(fused_P(h, l, true))));
  }
  h->fz_grid64 = std::min(fused_grid<cplx, false>(h->max_fiber, TSIZE, 0), need);
  h->fz_grid32 = std::min(h->fz_tcb32 > 0 ? fused_grid<cplxf, true>(h->max_fiber, h->fz_treg32, h->fz_tcb32)
                                          : fused_grid<cplxf, false>(h->max_fiber, h->fz_treg32 + h->fz_tregL32, 0),
                          need);
  {
    // PFMBEM_FUSED_GRID caps both grids (a test of the products on few blocks,
    // the group sizes of the batched launch; the cap is kept a multiple of 1)
    static const char* fg = std::getenv("PFMBEM_FUSED_GRID");
    if (fg && std::atoi(fg) > 0) {
      h->fz_grid64 = std::min(h->fz_grid64, std::atoi(fg));
      h->fz_grid32 = std::min(h->fz_grid32, std::atoi(fg));
    }
  }
  if (h->fz_grid64 <= 0 || h->fz_grid32 <= 0) return cudaSuccess;
  {
    // device-side GMRES steps: one block per SM (the steps are short; fewer
    // blocks keep the device-wide barriers cheap)
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (2 * (size_t)h->max_fiber + 512) * sizeof(cplx);
    int per32 = 0;
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(arnoldi_kernel<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(arnoldi_kernel<cplxf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, arnoldi_kernel<cplx>, FB, smem) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, arnoldi_kernel<cplxf>, FB, smem) == cudaSuccess &&
        per >= 1 && per32 >= 1)
      h->arn_grid = nsm;
    cudaGetLastError();
  }
  *ok = true;
  return cudaGetLastError();
}

cudaError_t k_fiber_symbols(pfmbem* h) {
  if (h->fz_nfft == 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)h->max_fiber * sizeof(cplx);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fiber_symbol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  prof_begin(h, PH_SETUP);
  fiber_symbol_kernel<<<h->fz_nfft, 256, smem, h->stream>>>(h->fz_fft, h->fib_off, h->fb_base, h->fb_val, h->fh_base,
                                                            h->tw, h->fh_val, h->fh_valf);
  prof_end(h, PH_SETUP);
  return cudaGetLastError();
}

cudaError_t k_precond_symbols(pfmbem* h) {
  if (h->fz_nfft == 0) return cudaSuccess;
  const size_t smem = 4 * (size_t)h->max_fiber * sizeof(cplx);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(precond_symbol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  prof_begin(h, PH_SETUP);
  precond_symbol_kernel<<<h->fz_nfft, 256, smem, h->stream>>>(h->fz_fft, h->fib_off, h->kt_base, h->kt_val,
                                                              h->fh_base, h->fh_val, h->eta, cplx{h->c2re, h->c2im},
                                                              h->tw, h->pc_val, h->pc_valf);
  prof_end(h, PH_SETUP);
  return cudaGetLastError();
}

cudaError_t k_precond_rows(pfmbem* h) {
  if (h->npr == 0) return cudaSuccess;
  const size_t smem = 9 * (size_t)h->max_fiber * sizeof(cplx);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(precond_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  prof_begin(h, PH_SETUP);
  precond_rows_kernel<<<h->npr, 256, smem, h->stream>>>(h->pr_list, h->fib_off, h->fb_base, h->fb_val, h->kt_base,
                                                        h->kt_val, h->eta, cplx{h->c2re, h->c2im}, h->pr_base,
                                                        h->pr_val, h->pr_valf);
  prof_end(h, PH_SETUP);
  return cudaGetLastError();
}

cudaError_t k_precond_apply(pfmbem* h, const cplx* x, cplx* y, int precision, const int* done) {
  const bool f32 = precision == PFMBEM_MIXED;
  const size_t smem = (2 * (size_t)h->max_fiber + 512) * (f32 ? sizeof(cplxf) : sizeof(cplx));
  prof_begin(h, PH_BLAS);
  if (f32) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(precond_apply_kernel<cplxf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    precond_apply_kernel<cplxf><<<h->M, 256, smem, h->stream>>>(h->M, h->fib_off, h->fh_base, h->pc_valf, h->twf,
                                                                h->pr_base, h->pr_valf, x, y, done,
                                                                2 * h->max_fiber);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(precond_apply_kernel<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    precond_apply_kernel<cplx><<<h->M, 256, smem, h->stream>>>(h->M, h->fib_off, h->fh_base, h->pc_val, h->tw,
                                                               h->pr_base, h->pr_val, x, y, done,
                                                               2 * h->max_fiber);
  }
  prof_end(h, PH_BLAS);
  return cudaGetLastError();
}

// One Arnoldi step of the device-side GMRES cycle (see arnoldi_kernel); with
// the preconditioner it also writes z_{j+1} = P^-1 v_{j+1} (in the precision of
// the products).
cudaError_t k_arnoldi_step(pfmbem* h, int j, int precision) {
  {
    cudaError_t e = reset_device_waits(h);
    if (e != cudaSuccess) return e;
  }
  GmresWork& g = h->gw;
  const bool f32 = precision == PFMBEM_MIXED;
  ArnArgs a{};
  if (h->pc && j + 1 < g.m) {
    a.Zn = g.Z + (size_t)(j + 1) * g.n;
    a.M = h->M;
    a.foff = h->fib_off;
    a.fh_base = h->fh_base;
    a.pc = f32 ? (const void*)h->pc_valf : (const void*)h->pc_val;
    a.tw = f32 ? (const void*)h->twf : (const void*)h->tw;
    a.pr_base = h->pr_base;
    a.pr = f32 ? (const void*)h->pr_valf : (const void*)h->pr_val;
    a.tws_off = 2 * h->max_fiber;
  }
  a.n = g.n;
  a.m = g.m;
  a.j = j;
  a.V = g.V;
  a.w = g.w;
  a.H = g.H;
  a.cs = g.cs;
  a.sn = g.sn;
  a.g = g.gv;
  a.acc = g.acc;
  a.ctl = g.ctl;
  a.ictl = g.ictl;
  a.bar = h->arn_bar;
  a.err = h->fz_err;
  void* args[] = {&a};
  const size_t smem = a.Zn ? (2 * (size_t)h->max_fiber + 512) * (f32 ? sizeof(cplxf) : sizeof(cplx)) : 0;
  const void* fn = f32 ? (const void*)arnoldi_kernel<cplxf> : (const void*)arnoldi_kernel<cplx>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  prof_begin(h, PH_BLAS);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(h->arn_grid), dim3(FB), args, smem, h->stream);
  prof_end(h, PH_BLAS);
  return e;
}

// y = R^{-1} g for the cycle's completed steps (device), for x += Z y.
cudaError_t k_arnoldi_solve(pfmbem* h, cplx* y) {
  GmresWork& g = h->gw;
  prof_begin(h, PH_BLAS);
  arnoldi_solve_kernel<<<1, 256, 0, h->stream>>>(g.H, g.gv, g.m, g.ictl, y);
  prof_end(h, PH_BLAS);
  return cudaGetLastError();
}

cudaError_t k_matvec_fused(pfmbem* h, const cplx* x, cplx* y, int precision, const int* done) {
  if (precision == PFMBEM_MIXED) return launch_fused<cplxf>(h, x, y, true, done);
  return launch_fused<cplx>(h, x, y, false, done);
}

#include "batch_solve.cuh"
