/*
 * pfmbem -- periodic fast-multipole BEM for acoustic transmission through a 2D
 * periodic array of fibers (Kress combined-layer formulation, quasi-periodic
 * along y), on one NVIDIA GB300 (sm_103a).
 *
 * Problem (paper Sec. 2): matrix wavenumber k in Omega_0, fiber wavenumber k1
 * inside the M fibers of one fundamental block, which repeats with period H
 * along y (h = (0, H), eq. 3, alpha = exp(i k H sin(theta))).  The incident wave
 * is exp(i k x.d), d = (cos theta, sin theta).  Unknowns are the double-layer
 * density phi and the single-layer density varphi on every fiber (eq. 4-5),
 * discretised as constants on the chords between consecutive boundary nodes
 * and collocated at the chord midpoints; the linear system is (I - A) Psi = B
 * of eq. 9 with Psi = (phi_1, varphi_1, ...) interleaved PER ELEMENT:
 *     Psi[2e] = phi_e,  Psi[2e+1] = varphi_e,   e = 0 .. E-1,
 * elements numbered fiber by fiber in node order.  Complex numbers are stored
 * as interleaved (re, im) doubles, so a complex vector of n entries is a
 * double array of 2n.
 *
 * Pointers: every data pointer may address host memory or device memory; the
 * library asks the CUDA runtime which, and stages host buffers through device
 * workspace with copies on the handle's stream.  Device buffers must belong to
 * the current device.  All GPU work is ordered on the stream given at create.
 *
 * Errors: every call returns a pfmbem_status; pfmbem_last_error(h) gives a
 * human-readable reason for the last failure on that handle.  Argument and
 * geometry errors are detected before any GPU work.  A handle is not
 * thread-safe; distinct handles are independent.
 */
#ifndef PFMBEM_H
#define PFMBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfmbem* pfmbem_t;

typedef enum {
  PFMBEM_OK = 0,
  PFMBEM_EINVAL = 1,    /* bad argument (null pointer, size, option out of range) */
  PFMBEM_EGEOM = 2,     /* bad geometry: degenerate element, clockwise fiber, block wider than 4 H */
  PFMBEM_EWOOD = 3,     /* too close to a Wood anomaly: min_n |kH(1 +- sin theta) - 2 pi n| < 1e-3 (Sec. 2) */
  PFMBEM_ENOMEM = 4,    /* device allocation failed */
  PFMBEM_ECUDA = 5,     /* a CUDA runtime call failed */
  PFMBEM_ENOCONV = 6,   /* GMRES stopped at maxit before reaching tol (best iterate is written) */
  PFMBEM_ETIMEOUT = 7,  /* a bounded device-side wait gave up (options.wait_us) */
  PFMBEM_ENUMERIC = 8   /* non-finite value detected (overflowing expansion tables, NaN residual) */
} pfmbem_status;

typedef enum { PFMBEM_SQUARE = 0, PFMBEM_HEXAGON = 1 } pfmbem_lattice;
typedef enum { PFMBEM_FP64 = 0, PFMBEM_MIXED = 1 } pfmbem_precision;

/* Options; a zero-initialised struct selects every default. */
typedef struct {
  int p;            /* expansion order at every level; 0 = per-level rule (below) */
  int p_min;        /* lower bound of the per-level rule; 0 = 24 (2p+1 = 49 coefficients;
                       the FMM's error on smooth densities falls by ~0.4 per order at
                       the fine levels and is ~1e-9 relative at 24) */
  double eta;       /* coupling constant eta of eq. 4 (a real number); 0 = k */
  int leaf_max;     /* target occupancy of a leaf box; 0 = 64 */
  int depth;        /* quadtree depth (levels 0..depth); 0 = chosen from leaf_max */
  int gmres_m;      /* GMRES restart length; 0 = 60 */
  int precision;    /* pfmbem_precision used by pfmbem_solve; default FP64 */
  int near_mode;    /* 0 = near-field and same-fiber element integrals computed once at
                       create and kept in device memory (default); 1 = recomputed in
                       every matvec (no cache memory) */
  int m2l_mode;     /* FP32 (mixed) M2L: 0 = default (CUDA cores, offset-grouped),
                       1 = CUDA cores, 2 = tensor cores (tcgen05, BF16 x3 split, FP32
                       accumulation in tensor memory) where 2(2p+1) <= 128 */
  int profile;      /* 1 = record per-phase CUDA-event times from create on (see pfmbem_profile) */
  int launch;       /* cached matvec: 0 = one cooperative launch per product with a
                       device-wide barrier between the stages (default; the tensor-core
                       M2L and devices without cooperative launch use 1); 1 = one kernel
                       per stage */
  int precond;      /* 0 = right block-Jacobi preconditioner over the fibers (default):
                       each fiber's same-fiber block of (I - A) (both wavenumbers, self
                       terms) inverted exactly by FFT where the fiber is a regular
                       polygon with 2^j elements, identity elsewhere; flexible GMRES.
                       1 = none */
  int wait_us;      /* bound of every device-side wait of the single-launch product, in
                       microseconds; 0 = one second.  A wait that runs out stops the
                       product, and the call that reads its result returns
                       PFMBEM_ETIMEOUT (the next product starts afresh) */
  int p_min_mixed;  /* lower bound of the per-level rule for the FP32 (mixed) product,
                       which uses the central sub-blocks of the FP64 tables; 0 = 18.
                       At most the FP64 order; the FP64 refinement of a mixed solve
                       keeps the solution at the FP64 product's accuracy */
  int batch_group;  /* blocks per instance group of pfmbem_solve_batch's persistent launch;
                       0 = 8 (raised to fit the coefficients of the tree's top level, one
                       warp each).  A batch uses the largest value among its handles */
  int tree;         /* 0 = square quadtree over the block (default); 1 = regular-triangle
                       quadtree for hexagon lattices (Sec. 3.1, Fig. 5): every fiber in the
                       hexagonal cell of its lattice point (the lattice below), the cell
                       split into six equilateral triangles and each triangle into four
                       down to the leaves; cells and triangles are neighbours when they
                       touch.  Its product is FP64, one kernel per stage, with the element
                       integrals cached at create (near_mode 0; M2M, M2L and L2L then in
                       double-float arithmetic, about 48 bits, on the FP32 pipes) or
                       computed in every product (near_mode 1); launch and m2l_mode must
                       be 0, a MIXED precision solves in FP64, and pfmbem_solve_batch
                       rejects it.
                       Default p_min 30.  EGEOM when a fiber leaves its cell, two fibers
                       share a cell or H is not a multiple (>= 2) of tri_a */
  double tri_a;     /* tree 1: nearest-neighbour spacing a of the hexagonal lattice, whose
                       lattice vectors are (0, a) and (a sqrt(3)/2, a/2) */
  double tri_ox, tri_oy;  /* tree 1: one point of that lattice */
} pfmbem_options;

/* Outcome of a solve. */
typedef struct {
  int iters;            /* total inner GMRES iterations (matrix-vector products) */
  int restarts;         /* GMRES restarts, or FP64 refinement steps in mixed mode */
  double rel_residual;  /* final true relative residual ||B - (I-A) Psi|| / ||B|| in FP64 */
  double ms;            /* wall time of the solve in milliseconds */
  int status;           /* pfmbem_status of the solve */
} pfmbem_info;

/* Plan summary for inspection and roofline accounting. */
typedef struct {
  int E;                  /* elements */
  int M;                  /* fibers */
  int depth;              /* quadtree depth */
  int p[16];              /* expansion order per level 0..depth */
  int nleaf_nonempty;     /* non-empty leaves */
  int64_t m2l_pairs;      /* (target box, source box) M2L translations per matvec, all levels */
  int64_t near_pairs;     /* (target element, source element) pairs of the near field */
  int64_t near_quad;      /* near-field kernel evaluations (pairs x Gauss nodes) per matvec */
  int64_t fiber_pairs;    /* same-fiber (k1) element pairs */
  int64_t fiber_quad;     /* same-fiber kernel evaluations per matvec */
  int p2m_nodes;          /* Gauss nodes per element in P2M */
  int lattice_q;          /* directly summed image rows in the lattice sums */
  double root_x0, root_y0;/* lower-left corner of the (first) root box (side H) */
  double setup_ms;        /* host wall time of pfmbem_create (the device part may still run) */
  int64_t near_blocks;    /* cached near-field 2x2 complex blocks (0 when not cached) */
  int64_t fiber_entries;  /* cached fiber-block complex entries (0 when not cached) */
  int cached;             /* 1 when the element integrals are cached in device memory */
  int tc_levels;          /* bit l set: the FP32 product runs level l's M2L on the tensor cores
                             (tcgen05, BF16x3 split products accumulated in FP32) */
  int p32[16];            /* expansion order per level of the FP32 product (<= p) */
  int64_t m2l_pairs_level[16];  /* M2L translations per matvec at each level 0..depth */
  int nroot;              /* root squares of side H in a row along x (1 unless the block is wider than H) */
  int super_p;            /* with nroot > 1: order of the super root over the row (0 otherwise) */
} pfmbem_plan_info;

/* Create a solver for one fundamental block (paper Sec. 2-3).
 *   M                 number of fibers (>= 1)
 *   nodes_per_fiber   [M] nodes of each fiber (>= 3), host or device
 *   nodes_xy          [sum N][2] boundary nodes, counter-clockwise per fiber
 *                     (outward normal = tangent turned clockwise, Sec. 2),
 *                     host or device, float64
 *   H                 period along y (paper H; "period L" elsewhere), > 0;
 *                     a block wider than H along x (up to 4 H) is covered by a
 *                     row of root squares of side H whose top operator couples
 *                     them (explicit root-to-root M2L for the near images, a
 *                     super root with the lattice sums for the far ones); such
 *                     blocks need the default product options (EINVAL otherwise)
 *   lattice           informational (square / hexagon; the quadtree is square)
 *   k, k1             matrix and fiber wavenumbers (> 0), k = omega/c_matrix
 *   rho_ratio         varrho = rho_matrix / rho_fiber of eq. 6 (> 0)
 *   theta             incidence angle in radians
 *   opt               options or NULL for defaults
 *   cuda_stream       cudaStream_t to order all work on (NULL = legacy stream)
 *   out               receives the handle; the handle owns all device state
 * Builds the quadtree (Sec. 3.1), self-element integrals, lattice sums
 * (Sec. 3.3) and translation tables.  Returns EGEOM/EWOOD/EINVAL/ENOMEM/ECUDA.
 * The device part of the set-up is queued on cuda_stream and the call returns
 * without waiting for it; the first later call on the handle that waits for
 * the stream (pfmbem_solve at its end, every other call at its start) returns
 * ENUMERIC if the set-up found a non-finite translation operator. */
pfmbem_status pfmbem_create(int M, const int* nodes_per_fiber, const double* nodes_xy,
                            double H, int lattice, double k, double k1, double rho_ratio,
                            double theta, const pfmbem_options* opt, void* cuda_stream,
                            pfmbem_t* out);

/* Release every resource of the handle (NULL is ignored). */
void pfmbem_destroy(pfmbem_t h);

/* Reason for the last failure on h (never NULL; "" if none). */
const char* pfmbem_last_error(pfmbem_t h);

/* Plan summary (sizes, orders, pair counts). */
pfmbem_status pfmbem_plan(pfmbem_t h, pfmbem_plan_info* info);

/* Right-hand side B of eq. 9 (complex [2E]):
 *   B[2e] = -u_inc(c_e),  B[2e+1] = (2i / (eta (1 + varrho))) du_inc/dnu(c_e). */
pfmbem_status pfmbem_rhs(pfmbem_t h, double* B);

/* y = (I - A) x, the operator of eq. 9, by the periodic FMM (Sec. 3) plus the
 * near field and the fiber-local k1 operators; x, y complex [2E]
 * (x and y must not overlap).  precision: PFMBEM_FP64 or PFMBEM_MIXED. */
pfmbem_status pfmbem_matvec(pfmbem_t h, const double* x, double* y, int precision);

/* Solve (I - A) Psi = B by restarted GMRES (Sec. 4: "GMRES"), right-preconditioned
 * by the fibers' inverse same-fiber blocks unless options.precond = 1 (flexible
 * GMRES: the preconditioned directions are kept).
 *   B     complex [2E] right-hand side, or NULL for the incident-wave B of eq. 9
 *   psi   complex [2E]; input initial guess if use_guess != 0, output solution
 *   tol   relative residual target (FP64 true residual)
 *   maxit maximum matrix-vector products
 * A guess x is first scaled by the gamma minimising ||B - gamma (I - A) x||
 * (one matvec: FP32 in mixed precision, whose residual only starts the
 * refinement, FP64 otherwise) and kept only if that residual is below ||B||;
 * otherwise the solve starts from zero.  In mixed precision the inner GMRES uses the
 * mixed matvec and an outer FP64 refinement loop restores FP64 accuracy.
 * Returns ENOCONV if tol is not met (psi still holds the best iterate).
 * info may be NULL. */
pfmbem_status pfmbem_solve(pfmbem_t h, const double* B, double* psi, int use_guess,
                           double tol, int maxit, pfmbem_info* info);

/* Solve many blocks together (band-gap sweeps, Sec. 4): the incident-wave
 * systems of ninst handles, each with its own geometry, size, frequency and
 * angle.  All instances are solved inside ONE persistent cooperative launch on
 * the first handle's stream (ordered after every handle's pending work): the
 * grid is cut into groups of blocks, and each group takes the next instance
 * from a device-side queue ordered by element count, longest first, and runs
 * its whole solve (refinement, GMRES cycles, products, Arnoldi steps) with
 * barriers over the group only.  The host waits once, at the end.  Handles
 * that cannot run in it (the tensor-core or per-stage product, restart length
 * above 250) make the whole batch run in host-driven lockstep instead, one unit
 * of GMRES work per instance per phase on the handles' own streams.  Each
 * handle uses its own precision: FP64, or mixed (FP32 operator in the inner
 * GMRES, FP64 residuals for the refinement).  psis[i] complex [2 E_i] (host or
 * device) receive the solutions; with use_guess != 0 they hold initial guesses
 * on entry (the learned warm start), each scaled by the gamma minimising
 * ||B - gamma (I - A) x|| and kept when that residual is below ||B|| (in mixed
 * precision gamma comes from the FP32 product; convergence is decided on FP64
 * residuals only).  infos may be NULL (info.ms is the batch's time).  Returns the first non-OK instance status (others are still solved);
 * ETIMEOUT for every instance when a bounded device wait of the launch gave up
 * (options.wait_us of the handles, 1 s by default). */
pfmbem_status pfmbem_solve_batch(int ninst, const pfmbem_t* hs, double* const* psis, int use_guess, double tol,
                                 int maxit, pfmbem_info* infos);

/* Scattered field u^s (eq. 7) at npts points outside the fibers, from the
 * densities psi: pts [npts][2] float64, u complex [npts]. */
pfmbem_status pfmbem_field(pfmbem_t h, const double* psi, int npts, const double* pts, double* u);

/* Scattered field u^s (eq. 7) and its derivative du^s/dx1 at npts points
 * outside the fibers (either output may be NULL, not both): pts [npts][2]
 * float64, u and dudx1 complex [npts].  Points must lie within (nroot/2 + 0.2) H
 * of the block centre along x, 0.7 H for one root (PFMBEM_EINVAL otherwise). */
pfmbem_status pfmbem_field_dx1(pfmbem_t h, const double* psi, int npts, const double* pts, double* u,
                               double* dudx1);

/* Energy transmission coefficient of Sec. 4 on the line x1 (normally the
 * block's right edge): ETC = (1/(kH)) int_0^H |du/dx1(x1, x2)| dx2 of the total
 * field u = u_inc + u^s, by the midpoint rule with npts points over one period
 * (the modulus is periodic along x2).  The modulus is not squared, as printed. */
pfmbem_status pfmbem_etc(pfmbem_t h, const double* psi, double x1, int npts, double* etc);

/* Bragg-order coefficients from the densities psi: for orders n with
 * |k sin(theta) + 2 pi n / H| < k, R_n (reflected, left of the block) and
 * T_n (transmitted, right; includes the incident wave for n = 0), plus the
 * energy sum E = sum (k_x,n / k_x,0)(|R_n|^2 + |T_n|^2).
 *   max_orders   capacity of orders/R/T; *norders receives the count.
 *   orders int[max_orders]; R, T complex [max_orders]; all host memory. */
pfmbem_status pfmbem_coefficients(pfmbem_t h, const double* psi, int max_orders, int* norders,
                                  int* orders, double* R, double* T, double* energy);

/* Lattice sums S_j = sum_{|m|>=2} alpha^m H_j(k|m|H) e^{i j theta_{-mh}} of
 * Sec. 3.3 (theta_{-mh} = -pi/2 for m > 0, +pi/2 for m < 0) for
 * j = -jmax .. jmax, computed as on the root translation: direct rows
 * 2 <= |m| <= q plus the two spectral tails integrated on the contour of eq. 18.
 * S complex [2 jmax + 1], index j + jmax. */
pfmbem_status pfmbem_lattice_sums(pfmbem_t h, int jmax, double* S);

/* ---------------------------------------------------------------------------
 * Learned warm start (beyond the paper: an AI-systems extension).  A small MLP
 * maps the block's parameters to the low Fourier modes of both densities on
 * every fiber; decoding them gives an initial guess for pfmbem_solve
 * (use_guess = 1).  The network is trained on the solver's own solutions.
 * --------------------------------------------------------------------------- */
typedef struct pfmbem_mlp* pfmbem_mlp_t;

/* MLP in -> hidden (GELU) x layers -> out (linear), FP32, weights drawn from a
 * counter-based generator (SplitMix64 of seed and parameter index) with
 * variance 1/fan_in, biases zero.  Parameters are one flat array: per layer W
 * [out][in] row-major, then b [out]. */
pfmbem_status pfmbem_mlp_create(int in, int hidden, int layers, int out, uint64_t seed, void* cuda_stream,
                                pfmbem_mlp_t* mlp);
void pfmbem_mlp_destroy(pfmbem_mlp_t mlp);
/* Parameter count; optionally copies them out (get) or in (set), host or device. */
pfmbem_status pfmbem_mlp_params(pfmbem_mlp_t mlp, int64_t* nparams, float* get, const float* set);
/* Y [batch][out] = MLP(X [batch][in]). */
pfmbem_status pfmbem_mlp_forward(pfmbem_mlp_t mlp, int batch, const float* X, float* Y);
/* Mean-squared error of MLP(X) against T [batch][out] (loss, host scalar, may be
 * NULL), its gradient with respect to the flat parameters (grad, may be NULL),
 * and, if lr > 0, one Adam step (beta1 0.9, beta2 0.999, eps 1e-8). */
pfmbem_status pfmbem_mlp_train(pfmbem_mlp_t mlp, int batch, const float* X, const float* T, float lr,
                               float* loss, float* grad);

/* Network input of the block: [kH/8, theta/(pi/2), per fiber ((cx-x0)/H,
 * (cy-y0)/H, 4r/H)] with (x0, y0) the root corner; x float [2 + 3M]. */
pfmbem_status pfmbem_warm_features(pfmbem_t h, float* x);
/* Per-fiber network input, one row of 5 + 3K floats per fiber (K <= 32):
 * [kH/8, theta/(pi/2), 4 r_i/H, (x_i - x_min)/H, (x_max - x_i)/H, then the K
 * nearest other fibers by distance, each (4 dx/H, 4 dy/H, 4 r_j/H) with dy to
 * the nearest periodic image, zeros where the block has fewer fibers].  x float
 * [M][5 + 3K]; a network on these rows maps one fiber's row to that fiber's
 * 2 x (2 nmodes + 1) complex modes (one row of pfmbem_warm_targets). */
pfmbem_status pfmbem_warm_features_local(pfmbem_t h, int K, float* x);
/* Fourier modes n = -nmodes..nmodes of both densities of every fiber of psi,
 * about the fiber centre, angles measured from the incidence direction, divided
 * by the incident phase at the centre:
 * t float [M][2][2 nmodes + 1][2] (re, im). */
pfmbem_status pfmbem_warm_targets(pfmbem_t h, int nmodes, const double* psi, float* t);
/* Inverse of pfmbem_warm_targets: psi0 complex [2E] from y (same layout). */
pfmbem_status pfmbem_warm_decode(pfmbem_t h, int nmodes, const float* y, double* psi0);

/* Kernel profiling (not part of the paper's method; measurement support).
 * Phases: 0 density gather, 1 P2M, 2 M2M, 3 M2L + L2L + root translation,
 * 4 L2P, 5 near-field P2P, 6 fiber-local P2P + combine, 7 GMRES vector
 * kernels, 8 set-up kernels, 9 output kernels (field, coefficients),
 * 10 element-integral cache build (the near-field and same-fiber Hankel
 * quadrature, once per create), 11 the single-launch matrix-vector product
 * (all of phases 0-6 in one cooperative kernel), 12 M2L where it runs apart
 * from L2L (the triangle tree's offset groups; phase 3 then holds L2L and the
 * operator between the cells); phases 0-6 and 11 of the FP32 (mixed)
 * matrix-vector product are counted at index + 16.
 * launches[] always counts the library's kernel launches; ms[] accumulates
 * CUDA-event device time per phase on the handle's stream while timing is on. */
typedef struct {
  double ms[32];
  int64_t launches[32];
  int64_t total_launches;
} pfmbem_profile_info;

/* enable_timing: 1 = record CUDA events around every launch; reset: 1 = zero counters. */
pfmbem_status pfmbem_profile(pfmbem_t h, int enable_timing, int reset);
/* Synchronises the stream and reads the counters. */
pfmbem_status pfmbem_profile_read(pfmbem_t h, pfmbem_profile_info* out);

/* Lattice sums without any device allocation (the paper has no counterpart;
 * this is a library convenience).  Some callers cannot call cudaMalloc:
 * plug-ins that run inside a host application which has already reserved the
 * device memory for its own pool or budget (a cudaMalloc there fails, or makes
 * the host release cached memory behind its back), and latency-critical loops
 * that must not enter the CUDA allocator, whose calls may synchronise the
 * device.  This entry point computes the same S_j as pfmbem_lattice_sums for
 * (k, H, theta) without a handle and without allocating: its device results go
 * to one fixed array of 129 complex numbers that is part of the library itself
 * (every GPU that loads the library holds it, 2 KiB, until the process exits).
 *   jmax    0 .. 128; larger values return PFMBEM_EINVAL
 *   S       complex [2 jmax + 1], index j + jmax, host or device memory; a
 *           device buffer must belong to the current device (PFMBEM_EINVAL
 *           otherwise, before any GPU work); with a device pointer the call
 *           only enqueues work on cuda_stream, with a host pointer it waits for
 *           the result
 * The first call on each device performs a one-time set-up there, with that
 * device current (copies the Gauss rules to the library's constant memory and
 * looks up the array's device address with cudaGetSymbolAddress); make that
 * first call before any stream capture begins.  Host threads that make their
 * first calls together run the set-up once.  All calls share the one array and
 * it keeps the last call's contents (each call clears what it accumulates into
 * before use), so calls whose GPU work overlaps (different streams or host
 * threads on the same device) race with each other: serialise them.
 * Returns EWOOD/EINVAL/ECUDA as pfmbem_create does. */
pfmbem_status pfmbem_lattice_sums_noalloc(double k, double H, double theta, int jmax, void* cuda_stream,
                                          double* S);

/* Measured arithmetic peak of the current device (measurement support, not
 * part of the paper's method): dtype 0 = FP64 FMA, 1 = FP32 FMA; TFLOP/s of
 * independent FMA chains over 8 CTAs per SM. */
pfmbem_status pfmbem_probe_peak(int dtype, double* tflops);

/* Self-element integrals used on the diagonal (flat element at its midpoint):
 * S_ee and the finite-part T_ee for k (out[0..1]) and k1 (out[2..3]) of every
 * element; out complex [E][4] in element order. */
pfmbem_status pfmbem_self_terms(pfmbem_t h, double* out);

#ifdef __cplusplus
}
#endif

#endif /* PFMBEM_H */
