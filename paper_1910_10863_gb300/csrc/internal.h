// Internal state of a pfmbem handle and the kernel launch interface shared by
// the host planner/driver (host.cpp) and the CUDA kernels (kernels.cu).
#pragma once

#include <algorithm>
#include <memory>
#include <utility>
#include <string>
#include <vector>

#include "common.cuh"

// Allocator whose value-less construct leaves the element uninitialised, so
// that resizing a byte buffer that is about to be overwritten does not first
// fill it with zeros.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
#include "../../include/pfmbem.h"

// One level of the uniform quadtree (level 0 = root box of side H).
struct Level {
  int p = 0, P = 0;          // order and coefficient count 2p+1
  int p32 = 0;               // order of the FP32 product's expansions (<= p; the central sub-blocks)
  double d = 0;              // box side
  double sigma = 0;          // expansion scale k * d / sqrt(2)
  std::vector<double> w;     // w_n = sigma^|n| / |n|!, n = -p..p (index n + p)
  double* w_dev = nullptr;   // device copy of w
  double* iw_dev = nullptr;  // 1 / w_n (device)
  int nbox = 0;              // 4^l boxes (Morton order)
  std::vector<int> hbegin, hend;   // element range of every box (sorted order)
  std::vector<int> hne;            // non-empty boxes
  // device
  cplx* M = nullptr;         // scaled multipoles [nbox][P]
  cplx* L = nullptr;         // scaled locals     [nbox][P]
  int* ne = nullptr;         // non-empty boxes
  int nne = 0;
  int* box_begin = nullptr;  // [nbox]
  int* box_end = nullptr;
  // M2L interaction lists (CSR over ne), entries: source box, offset id, image m
  int* il_ptr = nullptr;
  int* il_src = nullptr;
  int* il_off = nullptr;
  int* il_img = nullptr;
  int64_t nil = 0;
  // the same M2L pairs grouped by offset, in chunks of at most M2L_CHUNK pairs
  int* pr_tgt = nullptr;     // target box per pair
  int* pr_src = nullptr;     // source box per pair
  int* pr_img = nullptr;     // image m per pair
  int* pr_off = nullptr;     // offset id per pair
  int* ch_off = nullptr;     // offset id per chunk
  int* ch_beg = nullptr;     // first pair of the chunk
  int* ch_end = nullptr;     // one past the last pair
  int nchunk = 0;
  // tensor-core M2L: tiles of 128 target boxes, per tile the offsets present and
  // for every (tile, offset slot, target row) the source box (-1: none) and image
  int tc_ntile = 0;
  int* tc_box = nullptr;     // [ntile][128] target box (-1 padding)
  int* tc_noff = nullptr;    // [ntile]
  int* tc_offs = nullptr;    // [ntile][49]
  int* tc_src = nullptr;     // [ntile][49][128]
  int* tc_img = nullptr;     // [ntile][49][128]
  uint16_t* tc_B = nullptr;  // [49][3][kp][kp] BF16 parts of the real-embedded operators
  uint16_t* tc_Bf = nullptr; // the same for the single-launch FP32 product's central block (order p32)
  bool tc_fused = false;     // M2L of this level on tensor cores in the single-launch FP32 product
  cplx* m2l = nullptr;       // [49][P][P]: row = target coefficient, col = source coefficient
  cplx* m2lt = nullptr;      // the same operators transposed, [49][P source][P target]
  cplxf* m2ltf = nullptr;
  cplxf* m2ltl = nullptr;    // lo parts of m2lt: m2lt = m2ltf + m2ltl to ~48 bits (double-float M2L)
  // triangle tree: box centres, and per box the index of its M2M/L2L operator in
  // the parent level's tables (the children's offsets vary with the orientation)
  double2* ctr = nullptr;    // [nbox]
  int* pidx = nullptr;       // [nbox]
  int tri_noff = 0;          // distinct M2L offsets of the level
  cplxf* tri_m2l_hl = nullptr;   // hi, then lo parts of m2l ([2][tri_noff][P][P]) for the double-float M2L
  int tri_nop = 0;           // distinct child offsets below the level (M2M/L2L operators)
  cplxf* tri_m2m_hl = nullptr;   // hi, then lo parts of m2m and l2l ([2][tri_nop][P][P_child] each)
  cplxf* tri_l2l_hl = nullptr;
  cplx* m2m = nullptr;       // children (level l+1) -> this level: [4][P][P_child]
  cplx* l2l = nullptr;       // this level -> children: [4][P_child][P]
  // FP32 copies for the mixed path
  cplxf* Mf = nullptr;
  cplxf* Lf = nullptr;
  cplxf* m2lf = nullptr;
  cplxf* m2mf = nullptr;
  cplxf* m2ml = nullptr;     // lo parts of m2m (double-float M2M)
  cplxf* l2ll = nullptr;     // lo parts of l2l (double-float L2L)
  cplxf* l2lf = nullptr;
};

struct GmresWork {
  int n = 0, m = 0;
  cplx* V = nullptr;        // [(m+1)][n]
  cplx* w = nullptr;        // [n]
  cplx* r = nullptr;        // [n]
  cplx* x = nullptr;        // [n]
  cplx* b = nullptr;        // [n]
  cplx* d = nullptr;        // [n] FP64 residual of the refinement
  cplx* c = nullptr;        // [n] correction of the refinement
  cplx* Z = nullptr;        // [m][n] preconditioned basis (flexible GMRES)
  cplx* hcol = nullptr;     // [m+2] device dot results
  double* nrm = nullptr;    // [2]
  cplx* hhost = nullptr;    // pinned host mirror of hcol
  // device-side GMRES cycle (single-launch products only)
  cplx* H = nullptr;        // [(m+1)][m] rotated Hessenberg matrix
  cplx* cs = nullptr;       // [m] Givens rotations
  cplx* sn = nullptr;
  cplx* gv = nullptr;       // [m+1] rotated right-hand side
  cplx* acc = nullptr;      // [2][2 (m+1) + 1] CGS2 sums by step parity
  cplx* y = nullptr;        // [m] least-squares solution of the cycle
  double* ctl = nullptr;    // [4] estimate, ||b||, threshold
  int* ictl = nullptr;      // [4] done, steps completed, reason
};

enum Phase { PH_GATHER = 0, PH_P2M, PH_M2M, PH_LOCAL, PH_L2P, PH_NEAR, PH_FIBER, PH_BLAS, PH_SETUP, PH_OUT, PH_BUILD,
             PH_FUSED, PH_M2L, PH_COUNT };

// Launch counters and optional CUDA-event timing per phase.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;          // pool of events, used in begin/end pairs
  std::vector<int> phase_of_pair;       // phase of every recorded pair
  int used = 0;                         // events recorded since the last fold
  double ms[32] = {0};
  int64_t launches[32] = {0};
};

struct pfmbem {
  // problem (paper notation)
  int M = 0, E = 0, lattice = 0;
  double H = 0, k = 0, k1 = 0, rho = 0, theta = 0, eta = 0, beta = 0;
  cplx alpha{1, 0};
  double c2re = 0, c2im = 0;     // c2 = 2 / (i eta (1 + rho))
  pfmbem_options opt{};
  cudaStream_t stream = nullptr;
  int dev = -1;                  // device current at create (its streams come from that device's pool)
  cudaStream_t side = nullptr;   // second stream of the set-up: host planning overlaps the cache build
  cudaEvent_t side_ev = nullptr;
  cudaEvent_t pre_ev = nullptr;    // main-stream point the second stream waits for
  // set-up streams: lattice sums / P2M-L2P caches / near-field chain (high priority)
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t aux_ev[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ktab_ev = nullptr;  // the fiber k tables are built (near-field chain)
  cudaEvent_t fork_ev = nullptr;
  cudaStream_t astream = nullptr;  // stream of allocations and uploads while set-up runs on `side`
  std::string err;
  // plan
  int D = 0;
  int nroot = 1;                 // root squares of side H in a row along x (block width up to nroot H);
                                 // triangle tree: the hexagonal cells, one per fiber
  int tree = 0;                  // 0 = square quadtree, 1 = regular-triangle quadtree (hexagon lattices)
  bool tri_cache = false;        // triangle tree: element integrals and P2M/L2P coefficients cached
  double field_hw = 0;           // triangle tree: half the block's width along x (field point check)
  double x0 = 0, y0 = 0;
  Level lev[PF_MAXLEVEL + 1];
  int g_far = 4, g_far_f = 2;    // Gauss nodes per element in P2M (FP64 / FP32)
  int lattice_q = 8;
  pfmbem_plan_info info{};
  // elements, tree (sorted) order
  double2* s_c = nullptr;        // wrapped midpoint
  double2* s_t = nullptr;        // unit tangent
  double2* s_nu = nullptr;       // outward normal
  double* s_h = nullptr;         // length
  cplx* s_ph = nullptr;          // alpha^{-m0} input phase of the wrapped copy
  int* s_perm = nullptr;         // sorted -> original
  int* s_leaf = nullptr;         // leaf box (Morton) of every sorted element
  // elements, original order
  double2* o_c = nullptr;        // true midpoint
  double2* o_t = nullptr;
  double2* o_nu = nullptr;
  double* o_h = nullptr;
  int* o_fiber = nullptr;
  int* fib_off = nullptr;        // [M + 1]
  double* fib_geo = nullptr;     // [M][3] fiber centre (mean of nodes) and mean radius
  std::vector<double> hfib_geo;
  int* o_pos = nullptr;          // original -> sorted
  int* o_m0 = nullptr;           // original order: periods the element is shifted by when wrapped into the root
  int* o_key = nullptr;          // original order: leaf box (Morton) of the element
  cplx* self4 = nullptr;         // [E][4]: S_ee(k), T_ee(k), S_ee(k1), T_ee(k1)
  std::vector<int> hfib_off;
  int max_fiber = 0;
  // near lists over non-empty leaves (CSR): source leaf, image m
  int* nl_ptr = nullptr;
  int* nl_src = nullptr;
  int* nl_img = nullptr;
  // cached near field: per non-empty leaf, a dense [targets][sources] array of
  // 2x2 blocks (U' += a11 phi' + a12 varphi', dU' += a21 phi' + a22 varphi')
  bool cached = false;
  int64_t* nc_base = nullptr;    // [nleaf] value offset (in blocks) of the leaf
  int* nc_sbase = nullptr;       // [nleaf + 1] offset of the leaf's source list
  int* nc_src = nullptr;         // source element (sorted index) per list entry
  int* nc_img = nullptr;         // image m per list entry
  cplx* nc_val = nullptr;        // [blocks][4] FP64, formed on first use (k_near64)
  cplxf* nc_valf = nullptr;
  cplxf* nc_vall = nullptr;      // lo parts: nc_val = nc_valf + nc_vall to ~48 bits (double-float)
  int64_t nc_blocks = 0;
  int nc_maxns = 0;              // longest source list of a leaf
  int leaf_maxn = 0;             // most elements in a leaf
  // cached fiber blocks: the diagonal block of (I - A) of every fiber without
  // the FMM part (identity, k1 operators, self terms), row-major [2N][2N]
  int64_t* fb_base = nullptr;    // [M] offset of the fiber's block
  int* fb_circ = nullptr;        // [M] 1: regular polygon, circulant block stored as its row pair [2][2N]
  std::vector<int> hcirc;        // host copy of fb_circ
  int* fb_chunk = nullptr;       // [nchunk][3] = fiber, first row, last row + 1
  int* fb_rows = nullptr;        // elements whose row pairs are built (first element of a circulant fiber)
  // near-field integrals shared by translated copies of a fiber pair (lattices of identical fibers)
  int ntab = 0;                  // tables
  int64_t tab_entries = 0;
  int* tab_A = nullptr;          // [ntab] representative target fiber
  int* tab_B = nullptr;          // [ntab] representative source fiber
  int* tab_m = nullptr;          // [ntab] its image shift (periods)
  int64_t* tab_start = nullptr;  // [ntab + 1] first entry of every table (4 values each)
  int* tab_nb = nullptr;         // [ntab] elements of the source fiber
  cplx* tab_val = nullptr;       // as near-field blocks: (i/4) D, (eta/4) S, (i/4) T, (eta/4) K
  cplxf* tab_valf = nullptr;
  cplxf* tab_vall = nullptr;
  unsigned long long* nq = nullptr;   // near pairs left to integrate directly (leaf, row, column)
  unsigned* nq_len = nullptr;
  unsigned nq_cap = 0;
  int* pl_ptr = nullptr;         // [M + 1] per target fiber: (source fiber, image shift) -> table
  int* pl_fib = nullptr;
  int* pl_img = nullptr;
  int* pl_tab = nullptr;
  int nfb_rows = 0;
  int* s_m0 = nullptr;           // sorted: periods the element was shifted by when wrapped into the root
  int64_t* kt_base = nullptr;    // [M] first entry of the fiber's k table, -1 when not a regular polygon
  cplx* kt_val = nullptr;        // [sum N over regular fibers][4]: S, D, K, T at k of (f0, f0 + dl)
  cplx* kt_sval = nullptr;       // the same as near-field blocks: (i/4) D, (eta/4) S, (i/4) T, (eta/4) K
  cplxf* kt_svalf = nullptr;
  cplxf* kt_svall = nullptr;
  cplxf* dens_dd = nullptr;      // [2][2E] hi and lo parts of the sorted FP64 densities
  int nchunk = 0;
  cplx* fb_val = nullptr;
  cplxf* fb_valf = nullptr;
  int64_t fb_entries = 0;
  unsigned long long* stat_dev = nullptr;   // near pairs, near evaluations, fiber pairs, fiber evaluations
  // cached P2M / L2P operators, sorted element order: [E][2][P_leaf]
  //   P2M: M_n(leaf) = sum_f c[f][0][n] phi'_f + c[f][1][n] varphi'_f   (scaled by 1/w_n)
  //   L2P: U'_s = sum_l c[s][0][l] L_l(leaf), dU'_s = sum_l c[s][1][l] L_l(leaf)
  cplx* p2m_c = nullptr;
  cplx* l2p_c = nullptr;
  cplxf* p2m_cf = nullptr;
  cplxf* p2m_cl = nullptr;       // lo parts of p2m_c (double-float P2M)
  cplxf* l2p_cl = nullptr;       // lo parts of l2p_c (double-float L2P)
  cplxf* l2p_cf = nullptr;
  // FP32 work buffers of the mixed matvec
  int* tc_err = nullptr;         // set by the tensor-core M2L when a bounded wait gave up
  int* tab_err = nullptr;        // set when a translation table has a non-finite entry
  cplxf* densf = nullptr;        // [E][2]
  cplxf* Uf = nullptr;           // [E][2]
  // single-launch cached matvec (cooperative grid, device-wide barrier)
  bool fused = false;
  int fz_grid64 = 0, fz_grid32 = 0;
  int arn_grid = 0;              // blocks of the device-side GMRES step (0: host-side steps)
  unsigned long long* arn_bar = nullptr;   // its barrier's arrival counter
  unsigned long long* fz_bar = nullptr;    // [2] barrier arrival counters (FP64, FP32 product)
  unsigned long long* fz_arrive = nullptr; // diagnostic: [barrier][block] arrival times
  int fz_nfft = 0;               // fibers whose block-circulant block is applied by FFT
  int* fz_fft = nullptr;         // their indices
  int64_t* fh_base = nullptr;    // [M] first frequency of the fiber's block symbol (-1: none)
  cplx* fh_val = nullptr;        // [sum N][4] block symbols B^(r,s)(k)
  cplxf* fh_valf = nullptr;
  bool pc = false;               // block-Jacobi preconditioner available
  cplx* pc_val = nullptr;        // [sum N][4] inverse block symbols of the whole same-fiber blocks
  cplxf* pc_valf = nullptr;
  int npr = 0;                   // regular-polygon fibers whose element count is not 2^j
  int* pr_list = nullptr;
  int64_t* pr_base = nullptr;    // [M] their preconditioner row pairs (-1: none)
  cplx* pr_val = nullptr;        // [sum 4N]
  cplxf* pr_valf = nullptr;
  cplx* tw = nullptr;            // [512] e^{2 pi i j / 1024}
  cplxf* twf = nullptr;
  int fz_nchunk = 0;             // row chunks of the other fibers
  int* fz_chunk = nullptr;
  int* fz_err = nullptr;         // set when a bounded barrier wait gave up
  bool fz_dirty = false;         // fz_err was found set: clear the wait state before the next launch
  cplxf* fz_dlo = nullptr;       // [2E] lo parts of the FP32 product's sorted densities
  cplx* fz_rsum = nullptr;       // [E][4] FP64 row sums of the cached near blocks
  cplx* fz_frs = nullptr;        // [2E][2] FP64 row sums of the same-fiber rows applied by rows
  int* fz_rowfib = nullptr;      // [nrowsum][2] (fiber, row) of those rows
  int fz_nrowsum = 0;
  int fz_treg32 = 0;             // staged-operator region of the FP32 single-launch product (complex values)
  int fz_tregL32 = 0;            // its second region, for the L2L operators (0: none)
  size_t fz_tcb32 = 0;           // shared memory of the FP32 product's tensor-core M2L operands (0: none)
  int* s_li = nullptr;           // sorted element -> index of its leaf among the non-empty leaves
  int64_t* nr_meta = nullptr;    // [E][2] near-field row of a sorted element: block offset, (first source << 32) | sources
  int4* nr_piece = nullptr;      // near rows cut into pieces of <= 128 sources: first block offset (low,
                                 // high word), first source, (sources << 24) | element
  int nr_npiece = 0;
  cplx* Un = nullptr;            // [E][2] near-field part of (U', dU'), FP64 and FP32
  cplxf* Unf = nullptr;
  unsigned long long* fz_stamp = nullptr;   // [32] stage end times (diagnostic)
  cplx* root = nullptr;          // [P0][P0] periodic root translation ([nroot P0]^2 with several roots)
  // several roots: the super root (centre of the row, radius wide_rs, order
  // wide_ps) and the image row m0 from which its lattice sums take the images
  int wide_ps = 0, wide_m0 = 0;
  double wide_cx = 0, wide_cy = 0, wide_rs = 0;
  double* wide_w = nullptr;      // [Ps] weights of the super root's expansions
  cplx* wide_A = nullptr;        // [nroot][P0][Ps] M2M root j -> super root
  cplx* wide_B = nullptr;        // [nroot][Ps][P0] L2L super root -> root i
  cplx* wide_Rs = nullptr;       // [Ps][Ps] lattice-sum translation of the super root
  cplx* wide_ML = nullptr;       // [2][Ps] super multipole and local (field)
  cplxf* rootf = nullptr;
  cplx* rootc = nullptr;         // [4 P1][P0] root translation times the level-1 -> root M2M
  cplxf* rootcf = nullptr;
  cplx* m2m31 = nullptr;         // [P1][16 P3] level-3 -> level-1 M2M (two M2M steps in one)
  cplxf* m2m31f = nullptr;
  cplx* root1 = nullptr;         // [4][P1][4 P1] L(1) of each quadrant from the level-1 multipoles via the root
  cplxf* root1f = nullptr;
  // matvec work
  cplx* dens = nullptr;          // sorted [E][2] = (phi', varphi')
  cplx* U = nullptr;             // sorted [E][2] = (U', dU')
  cplx* stage_in = nullptr;      // [2E] staging for host buffers
  cplx* stage_out = nullptr;
  cplx* dev_rhs = nullptr;       // [2E]
  GmresWork gw;
  Prof prof;
  std::vector<void*> allocs;
  struct Carve {                 // the current chunk small arrays are carved from, per stream
    cudaStream_t stream = nullptr;
    unsigned char* base = nullptr;
    size_t used = 0, cap = 0;
  };
  std::vector<Carve> carves;
  int* hstat = nullptr;          // page-locked: the set-up's operator check, read back at create
  bool ready = true;             // the set-up has been waited for and its check reported
  // set-up trace (PFMBEM_TIMING=3): timing events recorded on the set-up streams
  bool trace_on = false;
  std::vector<const char*> trace_lbl;
  std::vector<cudaEvent_t> trace_ev;
  std::vector<double> trace_host;
  // batched table uploads during set-up (host.cpp upload / flush_uploads):
  // the open batch is written straight into the page-locked staging arena
  // when this create holds it, else (or once it overflows) into ub_buf
  bool ub_on = false;
  bool pin_user = false;           // counted among the users of the process-wide arena
  unsigned char* ub_pin = nullptr; // the arena, while this create holds it
  size_t ub_pin_cap = 0;
  size_t ub_pin_batch = 0;         // arena offset of the open batch
  size_t ub_len = 0;               // bytes of the open batch held in the arena
  bool ub_spill = false;           // the open batch moved to ub_buf
  std::vector<unsigned char, NoInitAlloc<unsigned char>> ub_buf;
  std::vector<std::pair<void**, size_t>> ub_fix;
  double setup_ms = 0;
};

// profiling hooks (kernels.cu)
void prof_begin(pfmbem* h, int phase);
void prof_end(pfmbem* h, int phase);
cudaError_t prof_fold(pfmbem* h);
void prof_release(pfmbem* h);
// outputs (kernels.cu): scattered field at points, Bragg-order coefficients
// tensor-core M2L (m2l_tc.cu)
int tc_kpad(int P);
cudaError_t k_tc_build_operator(pfmbem* h, int level);
cudaError_t k_tc_build_operator_fused(pfmbem* h, int level, int Pu);
cudaError_t k_m2l_tc(pfmbem* h, int level, const cplxf* M, cplxf* L);
cudaError_t k_build_caches(pfmbem* h, cudaEvent_t ktab_done = nullptr);
cudaError_t k_build_fiber_blocks(pfmbem* h);
cudaError_t k_near64(pfmbem* h);   // FP64 near blocks (hi + lo), formed on first use
// Diagnostic: records a timing event on st under label when the set-up trace is on.
void trace(pfmbem* h, cudaStream_t st, const char* label);
cudaError_t k_sort_elements(pfmbem* h);
// single-launch cached matvec (matvec_fused.cu)
cudaError_t k_fused_prepare(pfmbem* h, bool* ok);
cudaError_t k_top_operators(pfmbem* h, cudaStream_t st);
cudaError_t k_fused_tables(pfmbem* h);
cudaError_t k_matvec_fused(pfmbem* h, const cplx* x, cplx* y, int precision, const int* done = nullptr);
cudaError_t k_arnoldi_step(pfmbem* h, int j, int precision);
cudaError_t k_arnoldi_solve(pfmbem* h, cplx* y);
// Persistent batched solve: every instance solved inside one cooperative launch
// by groups of GS blocks, instances taken in the given order (longest first).
// cudaErrorNotSupported when an instance cannot run in it (see batch_eligible).
struct BatchResult {
  int iters, refinements, status;
  double relres;
};
bool batch_eligible(const pfmbem* h);
// Coefficients 2p + 1 of level l in the single-launch product of the given
// precision, and the levels (bit mask) whose FP32 M2L runs on the tensor cores.
int k_fused_order(const pfmbem* h, int l, bool f32);
int k_fused_tc_levels(const pfmbem* h);
cudaError_t k_batch_solve(int ninst, pfmbem* const* hs, const int* order, int GS, double tol, int maxit,
                          double trust_thr, int use_guess, cudaStream_t st, BatchResult* out, int* timed_out);
cudaError_t k_fiber_symbols(pfmbem* h);
cudaError_t k_precond_symbols(pfmbem* h);
cudaError_t k_precond_apply(pfmbem* h, const cplx* x, cplx* y, int precision, const int* done = nullptr);
cudaError_t k_precond_rows(pfmbem* h);
cudaError_t k_build_fmm_caches(pfmbem* h);
// learned warm start (mlp.cu)
cudaError_t k_warm_features(pfmbem* h, float* x_dev);
cudaError_t k_warm_features_local(pfmbem* h, int K, float* x_dev);
cudaError_t k_warm_targets(pfmbem* h, int nm, const cplx* psi, float* t_dev);
cudaError_t k_warm_decode(pfmbem* h, int nm, const float* y_dev, cplx* psi);
cudaError_t k_field_prepare(pfmbem* h, const cplx* psi);
cudaError_t k_coefficients(pfmbem* h, const cplx* psi, int norders, const int* orders_host, cplx* out_dev);

// ------------------------------------------------------------ kernel launches
void k_upload_gauss(const double* x, const double* w, const double* thr64, const double* thr32);
void k_upload_series();
cudaError_t k_self_terms(pfmbem* h);
// translation tables of all levels (kernels.cu)
struct TableLevels {
  int p[PF_MAXLEVEL + 1];
  double d[PF_MAXLEVEL + 1];
  const double* w[PF_MAXLEVEL + 1];
  cplx* T[PF_MAXLEVEL + 1];
  cplxf* Tf[PF_MAXLEVEL + 1];
  cplx* Tt[PF_MAXLEVEL + 1];
  cplxf* Ttf[PF_MAXLEVEL + 1];
  cplxf* Ttl[PF_MAXLEVEL + 1];
  cplx* A[PF_MAXLEVEL + 1];
  cplxf* Af[PF_MAXLEVEL + 1];
  cplxf* Al[PF_MAXLEVEL + 1];
  cplxf* Bl[PF_MAXLEVEL + 1];
  cplx* B[PF_MAXLEVEL + 1];
  cplxf* Bf[PF_MAXLEVEL + 1];
};
cudaError_t k_tables(pfmbem* h, const TableLevels& tl, cudaStream_t st);
cudaError_t k_root_operator(pfmbem* h, int p0, const double* w0, const cplx* S);
cudaError_t k_lattice_sums(pfmbem* h, int jmax, int q, cplx* out_dev, int mlo = 2);
// Blocks wider than H (a row of nroot root squares): the operator from every root's
// multipole to every root's local expansion, the images beyond the tree's lists
// included, into h->root ([nroot P0][nroot P0]), and the super root's operators
// kept for the field.
// nbr: optional [nroot][nroot][3] mask of the root pairs (i, j, image m = -1..1)
// that the tree's lists take (null: a row of squares, adjacent indices).
cudaError_t k_wide_top(pfmbem* h, const double2* dv, cplx* S, cplx* X, const unsigned char* nbr = nullptr);
// Triangle tree: level l's M2L operators for nm2l offsets (target - source
// centre) and its M2M/L2L operators for nshift child offsets (child - parent).
cudaError_t k_tri_tables(pfmbem* h, int l, const double2* m2l_v, int nm2l, const double2* shift_v, int nshift);
// Triangle tree: the cached FP64 product's tables (P2M/L2P coefficients at the
// leaves' centroids, near-field and same-fiber blocks).
cudaError_t k_tri_caches(pfmbem* h);
// Triangle tree: level l's M2L operator as hi and lo parts, and its M2L by
// offset groups in double-float arithmetic (matvec_fused.cu).
cudaError_t k_tri_m2l_split(pfmbem* h, int l);
cudaError_t k_tri_m2l_dd(pfmbem* h, int l);
// Triangle tree: M2M of level l from level l + 1, and L2L of level l from l - 1,
// in double-float arithmetic.
cudaError_t k_tri_m2m_dd(pfmbem* h, int l);
cudaError_t k_tri_l2l_dd(pfmbem* h, int l);
cudaError_t k_wide_local(pfmbem* h);
cudaError_t k_matvec(pfmbem* h, const cplx* x, cplx* y, int precision);
cudaError_t k_rhs(pfmbem* h, cplx* B);
cudaError_t k_field(pfmbem* h, const cplx* psi, int npts, const double2* pts, cplx* u, cplx* dudx1);
// BLAS-1 style helpers for GMRES (complex128, length n)
cudaError_t k_multidot(pfmbem* h, const cplx* V, int ncol, const cplx* w, int n, cplx* out);
cudaError_t k_gemv_sub(pfmbem* h, const cplx* V, int ncol, const cplx* coef, cplx* w, int n);
cudaError_t k_norm2(pfmbem* h, const cplx* v, int n, double* out);
cudaError_t k_scale_copy(pfmbem* h, const cplx* src, cplx s, cplx* dst, int n);
cudaError_t k_axpy(pfmbem* h, cplx a, const cplx* x, cplx* y, int n);   // y += a x
cudaError_t k_sub(pfmbem* h, const cplx* a, const cplx* b, cplx* out, int n);  // out = a - b
cudaError_t k_gemv_add(pfmbem* h, const cplx* V, int ncol, const cplx* coef, cplx* y, int n);  // y += V coef
