// Persistent batched solver: every instance of a band-gap sweep solved inside
// ONE cooperative launch.  Included at the end of matvec_fused.cu, whose
// single-launch product (fused_body), Arnoldi step (arnoldi_body) and
// preconditioner (precond_fiber) it runs.
//
// The grid is cut into groups of GS blocks.  A group takes the next instance
// from a device work counter over the instances sorted longest first (LPT
// order), runs the whole solve of that instance -- the FP64 iterative
// refinement around inner GMRES cycles on the FP32 product (mixed precision),
// or plain FP64 GMRES -- and then takes the next one.  The stages of a product
// and the steps of a cycle are separated by barriers over the group's GS blocks
// only (group_barrier on a counter of the group's own), so the instances run
// side by side with no host round trip and no device-wide barrier; control
// values (norms, residual estimates, step counts) are read back from global
// memory after a barrier by every block, which all take the same decisions.
// Reductions are summed in a fixed order over the group's blocks, so that
// every block sees the same value bit for bit.
//
// Every wait is bounded (wait_ns); a block whose wait ran out sets the error
// flag and leaves, and every other block leaves at its next barrier.

namespace {

// Per-instance state (device memory): the handle's GMRES workspace and the
// results, written by the group that solved the instance.
struct BatchInst {
  int n, m, M, pc, mixed, guess;     // guess: x holds an initial guess on entry
  cplx *b, *x, *d, *c, *w, *r, *V, *Z, *yv, *H, *gv, *acc;
  double* ctl;
  int* ictl;
  int iters, refinements, status, pad1;
  double relres;
};

struct BatchArgs {
  int ninst, GS;
  const int* order;                  // instances, longest first
  int* next;                         // work counter
  BatchInst* inst;
  const FusedArgs<cplxf>* fa32;      // [ninst] product arguments (x, y and the barrier set per product)
  const FusedArgs<cplx>* fa64;
  const ArnArgs* arn32;              // [ninst] Arnoldi-step arguments (j, Zn and the barrier set per step)
  const ArnArgs* arn64;
  unsigned long long* gbar;          // [groups] barrier counters
  int* gslot;                        // [groups] the group's current instance
  double* gpart;                     // [groups][2][4][GS] per-block partial sums
  int* err;                          // set when a bounded wait gave up
  unsigned long long wait_ns;
  double tol;
  double trust_thr;                  // estimate threshold (times tol) ending an inner cycle of the refinement
  int maxit;
  int fast_r1;                       // second refinement residual from the FP32 product
};

// Block b of the G blocks of one group.
struct Grp {
  int b, G;
  unsigned long long* bar;
  int* err;
  unsigned long long lim;
  double* part;                      // [2][4][G]
  int par;                           // slot set of the next group sum
};

__device__ __forceinline__ bool gsync(const Grp& g) { return group_barrier(g.bar, g.err, g.lim, g.G, g.b); }

// Sum of v over the threads of the block (every thread gets the same value).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
  return t;
}

// Sums over the group of K <= 4 values per block, in block order: each block
// writes its slots, a barrier, then every block adds the G slots of each value.
// The two slot sets alternate; a set is written again only two sums later, after
// a barrier that every block passes only once it has read the set.
__device__ bool group_sumv(Grp& g, const double* v, int K, double* out) {
  double* slot = g.part + (size_t)g.par * 4 * g.G;
  g.par ^= 1;
  if (threadIdx.x == 0)
    for (int q = 0; q < K; ++q) slot[q * g.G + g.b] = v[q];
  if (!gsync(g)) return false;
  for (int q = 0; q < K; ++q) {
    double t = 0;
    for (int i = 0; i < g.G; ++i) t += __ldcg(slot + q * g.G + i);
    out[q] = t;
  }
  return true;
}
__device__ __forceinline__ bool group_sum(Grp& g, double v, double* out) { return group_sumv(g, &v, 1, out); }

// Vector operations over the n entries, entry t by block (t / blockDim) mod G:
// every operation of the group gives an entry to the same block, so chains of
// them need no barrier in between.
#define GFOR(t, n) for (int t = g.b * (int)blockDim.x + (int)threadIdx.x; t < (n); t += g.G * (int)blockDim.x)

__device__ __forceinline__ void gfill0(const Grp& g, cplx* x, int n) { GFOR(t, n) x[t] = cplx{0, 0}; }
__device__ __forceinline__ void gcopy(const Grp& g, cplx* dst, const cplx* src, int n) { GFOR(t, n) dst[t] = src[t]; }
__device__ __forceinline__ void gscale_copy(const Grp& g, const cplx* src, double s, cplx* dst, int n) {
  GFOR(t, n) dst[t] = s * src[t];
}
__device__ __forceinline__ void gaxpy1(const Grp& g, const cplx* c, cplx* x, int n) { GFOR(t, n) x[t] += c[t]; }
// this block's part of ||v||^2
__device__ __forceinline__ double gnorm2_part(const Grp& g, const cplx* v, int n) {
  double s = 0;
  GFOR(t, n) s += abs2(v[t]);
  return block_sum(s);
}
// d = b - w; this block's part of ||d||^2
__device__ __forceinline__ double gsub_part(const Grp& g, const cplx* b, const cplx* w, cplx* d, int n) {
  double s = 0;
  GFOR(t, n) {
    const cplx v = b[t] - ldcg(w + t);
    d[t] = v;
    s += abs2(v);
  }
  return block_sum(s);
}
// x += sum_{c < k} Z_c y_c
__device__ __forceinline__ void ggemv_add(const Grp& g, const cplx* Z, int k, const cplx* y, cplx* x, int n) {
  __shared__ cplx s_y[ARN_MAXC];
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) s_y[i] = ldcg(y + i);
  __syncthreads();
  GFOR(t, n) {
    cplx v = x[t];
    for (int c = 0; c < k; ++c) v += ldcg(Z + (size_t)c * n + t) * s_y[c];
    x[t] = v;
  }
}

// The product and the Arnoldi step as functions of their own (not inlined into
// the persistent kernel, which keeps its compilation short).
template <class C>
__device__ __noinline__ bool fused_call(const FusedArgs<C>& a, int bid, int G) {
  return fused_body<C, false>(a, bid, G);
}
template <class C>
__device__ __noinline__ bool arnoldi_call(const ArnArgs& a, int b, int G, unsigned long long lim) {
  return arnoldi_body<C, true>(a, b, G, lim);
}

// y = A x by the group: the instance's arguments copied into this block's
// shared memory with x, y and the group's barrier in place; a group barrier at
// the end, after which y is complete.
template <class C>
__device__ bool gproduct(const FusedArgs<C>* src, const cplx* x, cplx* y, const Grp& g, unsigned long long* sargs) {
  static_assert(sizeof(FusedArgs<C>) % 8 == 0, "argument block in 8-byte words");
  constexpr int NW = (int)(sizeof(FusedArgs<C>) / 8);
  __syncthreads();
  const unsigned long long* s8 = reinterpret_cast<const unsigned long long*>(src);
  for (int i = threadIdx.x; i < NW; i += blockDim.x) sargs[i] = s8[i];
  __syncthreads();
  FusedArgs<C>* a = reinterpret_cast<FusedArgs<C>*>(sargs);
  if (threadIdx.x == 0) {
    a->x = x;
    a->y = y;
    a->bar = g.bar;
    a->err = g.err;
    a->wait_ns = g.lim;
  }
  __syncthreads();
  if (!fused_call<C>(*a, g.b, g.G)) return false;
  return gsync(g);
}

// Arnoldi step j of the cycle (w = A z_j in place), then a group barrier.
template <class C>
__device__ bool garnoldi(const ArnArgs* src, int j, cplx* Zn, const Grp& g, ArnArgs* sa) {
  __syncthreads();
  if (threadIdx.x == 0) {
    *sa = *src;
    sa->j = j;
    sa->Zn = Zn;
    sa->bar = g.bar;
    sa->err = g.err;
  }
  __syncthreads();
  if (!arnoldi_call<C>(*sa, g.b, g.G, g.lim)) return false;
  return gsync(g);
}

// y = P^-1 x by the group (the block-Jacobi preconditioner, a block per fiber).
template <class C>
__device__ void gprecond(const ArnArgs& a, const cplx* x, cplx* y, const Grp& g) {
  extern __shared__ __align__(128) unsigned char smraw[];
  C* xs = reinterpret_cast<C*>(smraw);
  C* tws = xs + a.tws_off;
  __syncthreads();
  if (g.b < a.M)
    for (int i = threadIdx.x; i < 512; i += blockDim.x) tws[i] = static_cast<const C*>(a.tw)[i];
  for (int fb = g.b; fb < a.M; fb += g.G) {
    __syncthreads();
    precond_fiber<C>(fb, a.foff, a.fh_base, static_cast<const C*>(a.pc), tws, a.pr_base,
                     static_cast<const C*>(a.pr), x, y, xs);
  }
  __syncthreads();
}

template <class C>
__device__ __forceinline__ const FusedArgs<C>* fargs(const BatchArgs& A, int ii);
template <>
__device__ __forceinline__ const FusedArgs<cplxf>* fargs<cplxf>(const BatchArgs& A, int ii) { return A.fa32 + ii; }
template <>
__device__ __forceinline__ const FusedArgs<cplx>* fargs<cplx>(const BatchArgs& A, int ii) { return A.fa64 + ii; }

struct GRes {
  int iters;
  double relres;
  int status;
};

// One restart cycle from V_0 (in place): the steps j < min(m, max_steps) as
// product + Arnoldi step until the step raises the done flag, then x += Z y
// (flexible) or V y.  As gmres_cycle_device on the host, with every decision
// taken on the device.
template <class C>
__device__ bool gcycle(const BatchArgs& A, int ii, Grp& g, cplx* x, double beta, double bnorm, double thr,
                       int max_steps, int* steps, double* est, int* reason, unsigned long long* sargs, ArnArgs* sarn) {
  const BatchInst& S = A.inst[ii];
  const int n = S.n, m = S.m;
  const ArnArgs* arn = sizeof(C) == sizeof(cplxf) ? A.arn32 + ii : A.arn64 + ii;
  if (g.b == 0) {
    const int nacc = 2 * (2 * (m + 1) + 1);
    for (int i = threadIdx.x; i <= m; i += blockDim.x) S.gv[i] = cplx{0, 0};
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) S.acc[i] = cplx{0, 0};
    __syncthreads();
    if (threadIdx.x == 0) {
      S.gv[0] = cplx{beta, 0};
      S.ctl[0] = 1.0;
      S.ctl[1] = bnorm;
      S.ctl[2] = thr;
      S.ictl[0] = S.ictl[1] = S.ictl[2] = S.ictl[3] = 0;
    }
  }
  if (S.pc) {
    if (!gsync(g)) return false;                 // V_0 complete
    gprecond<C>(*arn, S.V, S.Z, g);
  }
  if (!gsync(g)) return false;
  const int limit = min(m, max_steps);
  for (int j = 0; j < limit; ++j) {
    const cplx* zj = (S.pc ? S.Z : S.V) + (size_t)j * n;
    if (!gproduct<C>(fargs<C>(A, ii), zj, S.w, g, sargs)) return false;
    cplx* Zn = (S.pc && j + 1 < m) ? S.Z + (size_t)(j + 1) * n : nullptr;
    if (!garnoldi<C>(arn, j, Zn, g, sarn)) return false;
    if (__ldcg(S.ictl) != 0) break;
  }
  const int done = __ldcg(S.ictl);
  *reason = done ? __ldcg(S.ictl + 2) : 3;
  *steps = __ldcg(S.ictl + 1);
  *est = __ldcg(S.ctl);
  if (*steps > 0) {
    if (g.b == 0) arn_backsolve<true>(S.H, S.gv, m, *steps, S.yv);
    if (!gsync(g)) return false;
    ggemv_add(g, S.pc ? S.Z : S.V, *steps, S.yv, x, n);
    if (!gsync(g)) return false;
  }
  return true;
}

// Restarted GMRES(m) on b -> x in the precision C of the products (as gmres on
// the host): zero_start takes x = 0 without a product; trust_estimate ends at
// the first cycle whose Arnoldi estimate reached tol / 2; bnorm > 0 is ||b||.
template <class C>
__device__ bool gmres_dev(const BatchArgs& A, int ii, Grp& g, const cplx* b, cplx* x, double tol, int maxit,
                          bool zero_start, bool trust, double bnorm, GRes* res, unsigned long long* sargs,
                          ArnArgs* sarn) {
  const BatchInst& S = A.inst[ii];
  const int n = S.n;
  if (!(bnorm > 0)) {
    double s = 0;
    if (!group_sum(g, gnorm2_part(g, b, n), &s)) return false;
    bnorm = sqrt(s);
  }
  res->iters = 0;
  res->relres = 0;
  res->status = PFMBEM_OK;
  if (bnorm == 0) {
    gfill0(g, x, n);
    return gsync(g);
  }
  int iters = 0, restarts = 0;
  double relres = 1.0;
  bool done = false;
  while (!done) {
    double beta = bnorm;
    if (zero_start && restarts == 0) {
      gcopy(g, S.r, b, n);
    } else {
      if (!gproduct<C>(fargs<C>(A, ii), x, S.w, g, sargs)) return false;
      double s = 0;
      if (!group_sum(g, gsub_part(g, b, S.w, S.r, n), &s)) return false;
      beta = sqrt(s);
    }
    relres = beta / bnorm;
    if (!isfinite(relres)) {
      res->iters = iters;
      res->relres = relres;
      res->status = PFMBEM_ENUMERIC;
      return true;
    }
    if (relres <= tol || iters >= maxit) break;
    gscale_copy(g, S.r, 1.0 / beta, S.V, n);
    int steps = 0, reason = 0;
    double est = 1;
    if (!gcycle<C>(A, ii, g, x, beta, bnorm, (trust ? A.trust_thr : 0.5) * tol, maxit - iters, &steps, &est,
                   &reason, sargs, sarn))
      return false;
    iters += steps;
    ++restarts;
    if (steps == 0) break;
    if (reason != 3 && trust) {
      relres = est;
      done = true;
    }
  }
  res->iters = iters;
  res->relres = relres;
  res->status = relres <= tol ? PFMBEM_OK : PFMBEM_ENOCONV;
  return true;
}

// The whole solve of instance ii by the group, as pfmbem_solve (zero start):
// FP64 iterative refinement around inner GMRES on the FP32 product (mixed), or
// plain FP64 GMRES.  The results go to the instance's record.
__device__ bool solve_inst(const BatchArgs& A, int ii, Grp& g, unsigned long long* sargs, ArnArgs* sarn) {
  BatchInst& S = A.inst[ii];
  const int n = S.n, m = S.m;
  const double tol = A.tol;
  const int maxit = A.maxit;
  bool guess = S.guess != 0;
  if (!guess) gfill0(g, S.x, n);
  double bn2 = 0;
  if (!group_sum(g, gnorm2_part(g, S.b, n), &bn2)) return false;
  const double bn = sqrt(bn2);
  int iters = 0, refinements = 0, st = PFMBEM_ENOCONV;
  double relres = 0;
  // an initial guess x (the learned warm start): scaled by the gamma minimising
  // ||b - gamma A x||, kept when the scaled residual d = b - gamma A x is below
  // ||b||, else a zero start.  In mixed precision A x is the FP32 product: d only
  // starts the refinement, whose FP64 residuals decide convergence.
  double rn0 = bn2;
  bool g32 = false;
  if (bn > 0 && guess) {
    const bool ok = S.mixed ? gproduct<cplxf>(A.fa32 + ii, S.x, S.w, g, sargs)
                            : gproduct<cplx>(A.fa64 + ii, S.x, S.w, g, sargs);
    if (!ok) return false;
    double part[3] = {0, 0, 0}, tot[3];
    GFOR(t, n) {
      const cplx wv = ldcg(S.w + t), bv = S.b[t];
      part[0] += abs2(wv);
      part[1] += wv.re * bv.re + wv.im * bv.im;       // <w, b> = conj(w) b
      part[2] += wv.re * bv.im - wv.im * bv.re;
    }
    for (int q = 0; q < 3; ++q) part[q] = block_sum(part[q]);
    if (!group_sumv(g, part, 3, tot)) return false;
    const cplx gam = tot[0] > 0 ? cplx{tot[1] / tot[0], tot[2] / tot[0]} : cplx{0, 0};
    double dn = 0;
    GFOR(t, n) {
      const cplx v = S.b[t] - gam * ldcg(S.w + t);
      S.d[t] = v;
      S.x[t] = gam * S.x[t];
      dn += abs2(v);
    }
    if (!group_sum(g, block_sum(dn), &rn0)) return false;
    if (!(rn0 < bn2) || !isfinite(rn0)) {
      gfill0(g, S.x, n);
      guess = false;
      rn0 = bn2;
    }
    g32 = guess && S.mixed;
  }
  if (bn == 0) {
    st = PFMBEM_OK;
  } else if (S.mixed) {
    int stalls = 0;
    double prev = 1e300;
    relres = 1;
    for (; refinements < 50; ++refinements) {
      const bool r32 = refinements == 1 && A.fast_r1;
      double rn = bn2;
      if (refinements == 0 && guess) {
        rn = rn0;                          // d = b - gamma A x is in place
      } else if (refinements == 0) {
        gcopy(g, S.d, S.b, n);
      } else {
        const bool ok = r32 ? gproduct<cplxf>(A.fa32 + ii, S.x, S.w, g, sargs)
                            : gproduct<cplx>(A.fa64 + ii, S.x, S.w, g, sargs);
        if (!ok) return false;
        if (!group_sum(g, gsub_part(g, S.b, S.w, S.d, n), &rn)) return false;
      }
      relres = sqrt(rn) / bn;
      if (!isfinite(relres)) {
        st = PFMBEM_ENUMERIC;
        break;
      }
      if (relres <= tol && !r32 && !(refinements == 0 && g32)) {
        st = PFMBEM_OK;
        break;
      }
      if (iters >= maxit) break;
      if (!r32) {
        if (relres > 0.5 * prev) {
          if (++stalls >= 3) break;
        } else {
          stalls = 0;
        }
        prev = relres;
      }
      const double target = refinements == 0 ? fmax(1e-4, 0.3 * tol) : 0.3 * tol;
      const double inner_tol = fmax(1e-4, fmin(0.5, target / relres));
      const int cap = min(maxit - iters, 4 * m);
      gfill0(g, S.c, n);
      GRes r;
      if (!gmres_dev<cplxf>(A, ii, g, S.d, S.c, inner_tol, cap, true, true, sqrt(rn), &r, sargs, sarn))
        return false;
      if (r.status == PFMBEM_ENUMERIC) {
        st = PFMBEM_ENUMERIC;
        break;
      }
      iters += r.iters;
      gaxpy1(g, S.c, S.x, n);
      if (!gsync(g)) return false;
    }
    if (st != PFMBEM_OK && st != PFMBEM_ENUMERIC && iters < maxit) {
      // refinement stalled above tol: finish with FP64 GMRES from the iterate
      GRes r;
      if (!gmres_dev<cplx>(A, ii, g, S.b, S.x, tol, maxit - iters, false, false, bn, &r, sargs, sarn)) return false;
      st = r.status;
      iters += r.iters;
      relres = r.relres;
    }
  } else {
    GRes r;
    if (!gmres_dev<cplx>(A, ii, g, S.b, S.x, tol, maxit, !guess, false, bn, &r, sargs, sarn)) return false;
    st = r.status;
    iters = r.iters;
    relres = r.relres;
  }
  if (g.b == 0 && threadIdx.x == 0) {
    S.iters = iters;
    S.refinements = refinements;
    S.status = st;
    S.relres = relres;
  }
  return true;
}

constexpr int BATCH_ARGW = (int)((sizeof(FusedArgs<cplx>) > sizeof(FusedArgs<cplxf>) ? sizeof(FusedArgs<cplx>)
                                                                                      : sizeof(FusedArgs<cplxf>)) /
                                 8);

__global__ void __launch_bounds__(FB, 2) batch_solve_kernel(const __grid_constant__ BatchArgs A) {
  __shared__ __align__(16) unsigned long long s_args[BATCH_ARGW];
  __shared__ ArnArgs s_arn;
  const int grp = (int)blockIdx.x / A.GS;
  Grp g{(int)blockIdx.x - grp * A.GS, A.GS, A.gbar + grp, A.err, A.wait_ns, A.gpart + (size_t)grp * 8 * A.GS, 0};
  for (;;) {
    if (g.b == 0 && threadIdx.x == 0) A.gslot[grp] = atomicAdd(A.next, 1);
    if (!gsync(g)) return;
    const int q = __ldcg(A.gslot + grp);
    if (q >= A.ninst) return;
    if (!solve_inst(A, A.order[q], g, s_args, &s_arn)) return;
  }
}

#undef GFOR

// Host: arguments of instance h's products for the batched launch (groups of
// GS blocks, no tensor-core levels, the staging region of FP32 capped at the
// size of the FP64 one).
template <class C>
cudaError_t batch_fill(pfmbem* h, int GS, FusedArgs<C>& a) {
  cudaError_t e = fill_args<C>(h, nullptr, nullptr, nullptr, a);
  if (e != cudaSuccess) return e;
  const bool f32 = sizeof(C) == sizeof(cplxf);
  a.tc_any = 0;
  for (int l = 0; l <= PF_MAXLEVEL; ++l) a.tc_kp[l] = 0;
  if (f32) {
    const int cap = (int)((sizeof(cplx) * TSIZE) / sizeof(cplxf)) + FW * PF_NCOEF;
    a.treg = std::max(TSIZE, std::min(h->fz_treg32, cap));
    a.tregL = 0;
  }
  {
    const int nf = h->fz_nfft + h->fz_nchunk;
    const double wa = (double)h->lev[h->D].nne / FW;
    const int fb = (int)((double)GS * nf / (nf + wa) + 0.5);
    a.fblk = GS >= 16 ? std::max(1, std::min({fb, nf, GS - GS / 4})) : 0;
  }
  a.m2l_warp = f32 ? 0 : 1;
  a.near_first = 0;
  {
    const int64_t w = (int64_t)GS * FW;
    a.top3 = h->m2m31 != nullptr &&
             (int64_t)h->lev[2].nne * h->lev[2].P + (int64_t)h->lev[1].nne * h->lev[1].P + 4 * h->lev[0].P <= w;
  }
  a.stamp = nullptr;
  a.arrive = nullptr;
  a.bdone = nullptr;
  a.done = nullptr;
  return cudaSuccess;
}

ArnArgs batch_arn(pfmbem* h, bool f32) {
  GmresWork& g = h->gw;
  ArnArgs a{};
  if (h->pc) {
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
  a.V = g.V;
  a.w = g.w;
  a.H = g.H;
  a.cs = g.cs;
  a.sn = g.sn;
  a.g = g.gv;
  a.acc = g.acc;
  a.ctl = g.ctl;
  a.ictl = g.ictl;
  return a;
}

}  // namespace

int k_fused_order(const pfmbem* h, int l, bool f32) { return fused_P(h, l, f32); }

int k_fused_tc_levels(const pfmbem* h) {
  int mask = 0;
  for (int l = 1; l <= h->D; ++l) {
    const Level& L = h->lev[l];
    if (h->fz_tcb32 > 0 && L.tc_fused && L.tc_Bf && L.tc_ntile > 0 && tc::kpad(fused_P(h, l, true)) <= TC_KPMAX)
      mask |= 1 << l;
  }
  return mask;
}

// Can handle h run in the persistent batched launch?  (single-launch products,
// device-side GMRES workspace, no tensor-core M2L levels)
bool batch_eligible(const pfmbem* h) {
  return h && h->fused && h->cached && h->arn_grid > 0 && h->fz_tcb32 == 0 && h->gw.V && h->gw.H &&
         h->gw.m < ARN_MAXC;
}

// Dynamic shared memory of the batched launch for instance h.
static size_t batch_smem(const pfmbem* h) {
  const size_t f64 = fused_smem<cplx>(h->max_fiber, TSIZE, 0, FW);
  const size_t pcb = (2 * (size_t)h->max_fiber + 512) * sizeof(cplx);
  const size_t arn = (size_t)std::max(2 * ARN_MAXC, 32 * 32 + 32) * sizeof(cplx);   // rotations; back substitution
  return std::max({f64, pcb, arn});
}

cudaError_t k_batch_solve(int ninst, pfmbem* const* hs, const int* order, int GS, double tol, int maxit,
                          double trust_thr, int use_guess, cudaStream_t st, BatchResult* out, int* timed_out) {
  *timed_out = 0;
  if (ninst <= 0) return cudaSuccess;
  if (GS < 1) return cudaErrorInvalidValue;
  for (int i = 0; i < ninst; ++i)
    if (!batch_eligible(hs[i])) return cudaErrorNotSupported;
  // groups large enough for the root's coefficients, one warp each
  for (int i = 0; i < ninst; ++i) GS = std::max(GS, (hs[i]->lev[0].nne * hs[i]->lev[0].P + FW - 1) / FW);
  size_t smem = 0;
  for (int i = 0; i < ninst; ++i) smem = std::max(smem, batch_smem(hs[i]));
  const void* fn = (const void*)batch_solve_kernel;
  {
    static std::atomic<size_t> set_max{0};
    size_t cur = set_max.load();
    if (smem > cur) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      while (smem > cur && !set_max.compare_exchange_weak(cur, smem)) {
      }
    }
  }
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, FB, smem);
    if (e != cudaSuccess) return e;
  }
  if (per < 1) return cudaErrorNotSupported;
  int ngroup = (nsm * std::min(per, 2)) / GS;
  ngroup = std::min(ngroup, ninst);
  if (ngroup < 1) return cudaErrorNotSupported;
  const int grid = ngroup * GS;
  // the batch's argument block: one upload of one host buffer
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_inst = 0;
  const size_t o_fa32 = al(o_inst + sizeof(BatchInst) * ninst);
  const size_t o_fa64 = al(o_fa32 + sizeof(FusedArgs<cplxf>) * ninst);
  const size_t o_a32 = al(o_fa64 + sizeof(FusedArgs<cplx>) * ninst);
  const size_t o_a64 = al(o_a32 + sizeof(ArnArgs) * ninst);
  const size_t o_ord = al(o_a64 + sizeof(ArnArgs) * ninst);
  const size_t o_bar = al(o_ord + sizeof(int) * ninst);
  const size_t o_slot = al(o_bar + sizeof(unsigned long long) * ngroup);
  const size_t o_part = al(o_slot + sizeof(int) * ngroup);
  const size_t o_next = al(o_part + sizeof(double) * 8 * grid);
  const size_t o_err = o_next + 16;
  const size_t total = al(o_err + 16);
  std::vector<unsigned char> hb(total, 0);
  BatchInst* bi = reinterpret_cast<BatchInst*>(hb.data() + o_inst);
  FusedArgs<cplxf>* f32 = reinterpret_cast<FusedArgs<cplxf>*>(hb.data() + o_fa32);
  FusedArgs<cplx>* f64 = reinterpret_cast<FusedArgs<cplx>*>(hb.data() + o_fa64);
  ArnArgs* a32 = reinterpret_cast<ArnArgs*>(hb.data() + o_a32);
  ArnArgs* a64 = reinterpret_cast<ArnArgs*>(hb.data() + o_a64);
  std::memcpy(hb.data() + o_ord, order, sizeof(int) * ninst);
  unsigned long long wait_ns = 1000000000ull;
  for (int i = 0; i < ninst; ++i) {
    pfmbem* h = hs[i];
    GmresWork& gw = h->gw;
    cudaError_t e = batch_fill<cplxf>(h, GS, f32[i]);
    if (e == cudaSuccess) e = batch_fill<cplx>(h, GS, f64[i]);
    if (e != cudaSuccess) return e;
    a32[i] = batch_arn(h, true);
    a64[i] = batch_arn(h, false);
    BatchInst& b = bi[i];
    b.n = gw.n;
    b.m = gw.m;
    b.M = h->M;
    b.pc = h->pc ? 1 : 0;
    b.mixed = h->opt.precision == PFMBEM_MIXED ? 1 : 0;
    b.b = gw.b; b.x = gw.x; b.d = gw.d; b.c = gw.c; b.w = gw.w; b.r = gw.r; b.V = gw.V; b.Z = gw.Z;
    b.yv = gw.y; b.H = gw.H; b.gv = gw.gv; b.acc = gw.acc; b.ctl = gw.ctl; b.ictl = gw.ictl;
    b.status = PFMBEM_ENOCONV;
    b.guess = use_guess ? 1 : 0;
    if (h->opt.wait_us > 0) wait_ns = std::min(wait_ns, 1000ull * (unsigned long long)h->opt.wait_us);
  }
  // the launch is ordered after every handle's pending work on its own stream
  // (set-up tails, right-hand sides, and what the argument fills just queued)
  for (int i = 0; i < ninst; ++i) {
    if (hs[i]->stream == st) continue;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, hs[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return e;
  }
  unsigned char* db = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&db), total, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(db, hb.data(), total, cudaMemcpyHostToDevice, st);
  BatchArgs A{};
  A.ninst = ninst;
  A.GS = GS;
  A.order = reinterpret_cast<const int*>(db + o_ord);
  A.next = reinterpret_cast<int*>(db + o_next);
  A.inst = reinterpret_cast<BatchInst*>(db + o_inst);
  A.fa32 = reinterpret_cast<const FusedArgs<cplxf>*>(db + o_fa32);
  A.fa64 = reinterpret_cast<const FusedArgs<cplx>*>(db + o_fa64);
  A.arn32 = reinterpret_cast<const ArnArgs*>(db + o_a32);
  A.arn64 = reinterpret_cast<const ArnArgs*>(db + o_a64);
  A.gbar = reinterpret_cast<unsigned long long*>(db + o_bar);
  A.gslot = reinterpret_cast<int*>(db + o_slot);
  A.gpart = reinterpret_cast<double*>(db + o_part);
  A.err = reinterpret_cast<int*>(db + o_err);
  A.wait_ns = wait_ns;
  A.tol = tol;
  A.trust_thr = trust_thr;
  A.maxit = maxit;
  static const bool r1_fp64 = std::getenv("PFMBEM_R1_FP64") != nullptr;
  A.fast_r1 = r1_fp64 ? 0 : 1;
  if (e == cudaSuccess) {
    void* args[] = {&A};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(FB), args, smem, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb.data(), db, o_fa32, cudaMemcpyDeviceToHost, st);           // the instance records
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data() + o_err, db + o_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(db, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *timed_out = *reinterpret_cast<int*>(hb.data() + o_err);
  for (int i = 0; i < ninst; ++i) {
    out[i].iters = bi[i].iters;
    out[i].refinements = bi[i].refinements;
    out[i].status = bi[i].status;
    out[i].relres = bi[i].relres;
  }
  return cudaSuccess;
}
