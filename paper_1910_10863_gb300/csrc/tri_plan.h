// Regular-triangle quadtree for hexagon lattices (Sec. 3.1, Fig. 5), included by
// host.cpp (it uses the planner's upload and allocation helpers).
//
// Every fiber sits in the hexagonal (Voronoi) cell of its point of the hexagonal
// lattice: nearest-neighbour spacing a, one lattice vector along y.  The cell
// (level 0, circumradius a / sqrt 3) is split into six equilateral triangles
// (level 1), each of those into four (the three corner triangles and the
// inverted middle one), and so on.  Boxes are numbered so that a level-1 box is
// 6 i + s (cell i, sector s) and a box below is 4 b + q (parent b, child q); the
// centre of a triangle is its centroid, of a cell its lattice point.
//
// Two cells or two triangles of one level are neighbours when they touch (share
// a vertex, counting the images m = -1, 0, 1 of the y-period; Sec. 3.1: adjacent
// basic trees share a vertex).  A target's M2L sources are the children of its
// parent's neighbours that do not touch it; the leaves' neighbours form the near
// field.  Cells that do not touch, and every image |m| >= 2, interact at level 0
// through one operator between all cells: explicit M2L for the images
// |m| < m0 and a super root over the block whose lattice sums (Sec. 3.3) take
// the images |m| >= m0 (the operator of the blocks wider than H, k_wide_top).
//
// The tree drives an FP64 product, the single solve and the outputs.  The
// product applies tables built once here where they do not depend on the tree's
// shape (near-field and same-fiber blocks, P2M/L2P coefficients at the leaves'
// centroids, M2L by offset groups); with near_mode 1 it integrates the element
// integrals in every product instead.  The mixed-precision single-launch
// products and the batched solver stay with the square tree.

struct TriBox {
  double2 v[3];
};

static inline double2 tri_mid(double2 a, double2 b) { return double2{0.5 * (a.x + b.x), 0.5 * (a.y + b.y)}; }

// Child q of triangle (A, B, C): the corners A, B, C, then the middle triangle.
static inline TriBox tri_child(const TriBox& t, int q) {
  const double2 A = t.v[0], B = t.v[1], C = t.v[2];
  const double2 AB = tri_mid(A, B), BC = tri_mid(B, C), CA = tri_mid(C, A);
  switch (q) {
    case 0: return TriBox{{A, AB, CA}};
    case 1: return TriBox{{AB, B, BC}};
    case 2: return TriBox{{CA, BC, C}};
    default: return TriBox{{BC, CA, AB}};
  }
}

// The child of triangle t that holds point x: a corner when x's barycentric
// coordinate of that vertex is at least 1/2, else the middle triangle.
static inline int tri_locate(const TriBox& t, double2 x) {
  const double2 A = t.v[0], B = t.v[1], C = t.v[2];
  const double det = (B.x - A.x) * (C.y - A.y) - (C.x - A.x) * (B.y - A.y);
  const double lb = ((x.x - A.x) * (C.y - A.y) - (C.x - A.x) * (x.y - A.y)) / det;
  const double lc = ((B.x - A.x) * (x.y - A.y) - (x.x - A.x) * (B.y - A.y)) / det;
  const double la = 1.0 - lb - lc;
  if (la >= 0.5) return 0;
  if (lb >= 0.5) return 1;
  if (lc >= 0.5) return 2;
  return 3;
}

static inline double2 tri_centroid(const TriBox& t) {
  return double2{(t.v[0].x + t.v[1].x + t.v[2].x) / 3.0, (t.v[0].y + t.v[1].y + t.v[2].y) / 3.0};
}

// Vertex-sharing test of two triangles of one tiling level (tol: a small
// fraction of the side), the second shifted by dy along y.
static inline bool tri_touch(const TriBox& a, const TriBox& b, double dy, double tol) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (std::fabs(a.v[i].x - b.v[j].x) < tol && std::fabs(a.v[i].y - b.v[j].y - dy) < tol) return true;
  return false;
}

// Index of offset v in a level's table of distinct offsets (quantum: a small
// fraction of the level's side), appended when new.
struct OffsetTable {
  double quantum = 1.0;
  std::map<std::pair<long long, long long>, int> idx;
  std::vector<double2> v;
  int get(double2 o) {
    const auto key = std::make_pair(std::llround(o.x / quantum), std::llround(o.y / quantum));
    auto it = idx.find(key);
    if (it != idx.end()) return it->second;
    const int i = (int)v.size();
    idx.emplace(key, i);
    v.push_back(o);
    return i;
  }
};

static pfmbem_status build_plan_tri(pfmbem* h, const double* nodes, const std::vector<int>& foff,
                                    const std::vector<double2>& c,
                                    const std::vector<double2>& t, const std::vector<double2>& nu,
                                    const std::vector<double>& len, const std::vector<int>& fib, double hmax,
                                    double t0) {
  const int M = h->M, E = h->E;
  const double H = h->H, k = h->k;
  const double a = h->opt.tri_a, ox = h->opt.tri_ox, oy = h->opt.tri_oy;
  if (!(a > 0) || !std::isfinite(ox) || !std::isfinite(oy))
    return fail(h, PFMBEM_EINVAL, "triangle tree: the lattice spacing tri_a must be positive, tri_ox/tri_oy finite");
  if (h->opt.launch != 0 || h->opt.m2l_mode == 2)
    return fail(h, PFMBEM_EINVAL, "triangle tree: runs its own FP64 product (launch and m2l_mode must be 0)");
  const int nH = (int)std::lround(H / a);
  if (nH < 2 || std::fabs(H / a - nH) > 1e-9 * (H / a))
    return fail(h, PFMBEM_EGEOM, "triangle tree: the period H must be a multiple (>= 2) of the lattice spacing");
  if (0.5 * k * hmax > 4.0) return fail(h, PFMBEM_EINVAL, "elements longer than 8/k");
  h->tree = 1;
  h->cached = false;
  h->fused = false;
  h->ub_on = true;                 // tables below go up in a few batched copies
  pin_acquire(h);
  const double s3 = std::sqrt(3.0);
  const double r0 = a / s3;                               // circumradius of a cell
  const double2 e1{0.0, a}, e2{0.5 * s3 * a, 0.5 * a};   // lattice vectors
  // ---------------------------------------------------- cells: the lattice point of every fiber
  std::vector<double2> C(M);
  {
    std::map<std::pair<long long, long long>, int> seen;
    for (int i = 0; i < M; ++i) {
      const double dx = h->hfib_geo[3 * i] - ox, dy = h->hfib_geo[3 * i + 1] - oy;
      const double v = dx / e2.x, u = (dy - v * e2.y) / a;
      double best = 1e300;
      long long bu = 0, bv = 0;
      for (long long vv = (long long)std::floor(v) - 1; vv <= (long long)std::floor(v) + 2; ++vv)
        for (long long uu = (long long)std::floor(u) - 1; uu <= (long long)std::floor(u) + 2; ++uu) {
          const double px = ox + vv * e2.x, py = oy + uu * a + vv * e2.y;
          const double d2 = (px - ox - dx) * (px - ox - dx) + (py - oy - dy) * (py - oy - dy);
          if (d2 < best) { best = d2; bu = uu; bv = vv; }
        }
      C[i] = double2{ox + bv * e2.x, oy + bu * e1.y + bv * e2.y};
      // one fiber per cell, also modulo the period
      const long long uw = ((bu % nH) + nH) % nH;   // index along e1 = (0, a), wrapped by the period
      if (!seen.emplace(std::make_pair(uw, bv), i).second)
        return fail(h, PFMBEM_EGEOM, "triangle tree: two fibers in one lattice cell (modulo the period)");
      // every node inside the cell: |(x - C) . n| < a / 2 for the edge normals at 30, 90, 150 degrees
      for (int j = foff[i]; j < foff[i + 1]; ++j) {
        const double* p = nodes + 2 * (size_t)j;
        const double qx = p[0] - C[i].x, qy = p[1] - C[i].y;
        for (int e = 0; e < 3; ++e) {
          const double ang = M_PI / 6 + e * M_PI / 3;
          if (std::fabs(qx * std::cos(ang) + qy * std::sin(ang)) >= 0.5 * a * (1 - 1e-12))
            return fail(h, PFMBEM_EGEOM, "triangle tree: fiber " + std::to_string(i) + " leaves its hexagonal cell");
        }
      }
    }
  }
  // ---------------------------------------------------- element paths down the tree
  constexpr int kDmax = 8;
  std::vector<unsigned char> path((size_t)E * (kDmax + 1), 0);   // sector at level 1, child q below
  for (int e = 0; e < E; ++e) {
    const int i = fib[e];
    double ang = std::atan2(c[e].y - C[i].y, c[e].x - C[i].x);
    if (ang < 0) ang += 2 * M_PI;
    const int s = std::min(5, std::max(0, (int)std::floor(ang / (M_PI / 3))));
    TriBox tb{{C[i], double2{C[i].x + r0 * std::cos(s * M_PI / 3), C[i].y + r0 * std::sin(s * M_PI / 3)},
               double2{C[i].x + r0 * std::cos((s + 1) * M_PI / 3), C[i].y + r0 * std::sin((s + 1) * M_PI / 3)}}};
    path[(size_t)e * (kDmax + 1) + 1] = (unsigned char)s;
    for (int l = 2; l <= kDmax; ++l) {
      const int q = tri_locate(tb, c[e]);
      path[(size_t)e * (kDmax + 1) + l] = (unsigned char)q;
      tb = tri_child(tb, q);
    }
  }
  auto key_at = [&](int e, int l) {
    int b = fib[e];
    if (l >= 1) b = 6 * b + path[(size_t)e * (kDmax + 1) + 1];
    for (int j = 2; j <= l; ++j) b = 4 * b + path[(size_t)e * (kDmax + 1) + j];
    return b;
  };
  auto nbox_at = [&](int l) { return l == 0 ? (size_t)M : (size_t)6 * M << (2 * (l - 1)); };
  // ---------------------------------------------------- depth
  const int leaf_max = h->opt.leaf_max > 0 ? h->opt.leaf_max : 64;
  int D = h->opt.depth;
  if (D <= 0) {
    for (D = 1; D < kDmax; ++D) {
      std::vector<int> cnt(nbox_at(D), 0);
      int mx = 0;
      for (int e = 0; e < E; ++e) mx = std::max(mx, ++cnt[key_at(e, D)]);
      if (mx <= leaf_max) break;
    }
  }
  if (D < 1 || D > kDmax) return fail(h, PFMBEM_EINVAL, "triangle tree: depth must be in [1, 8]");
  // (every level keeps expansions for all its boxes: at most 4 M leaves, about
  // 4 GB of FP64 multipoles and locals at p 30)
  if (nbox_at(D) > ((size_t)1 << 22)) return fail(h, PFMBEM_EINVAL, "triangle tree: too many boxes at this depth");
  h->D = D;
  // ---------------------------------------------------- sort by leaf (stable counting sort)
  std::vector<int> key(E), perm(E), pos(E);
  for (int e = 0; e < E; ++e) key[e] = key_at(e, D);
  {
    std::vector<int> start(nbox_at(D) + 1, 0);
    for (int e = 0; e < E; ++e) start[key[e] + 1]++;
    for (size_t b = 0; b + 1 < start.size(); ++b) start[b + 1] += start[b];
    for (int e = 0; e < E; ++e) perm[start[key[e]]++] = e;
  }
  for (int s = 0; s < E; ++s) pos[perm[s]] = s;
  // ---------------------------------------------------- levels: geometry, ranges, orders
  std::vector<std::vector<TriBox>> geo(D + 1);
  std::vector<std::vector<double2>> ctr(D + 1);
  ctr[0] = C;
  for (int l = 1; l <= D; ++l) {
    geo[l].resize(nbox_at(l));
    ctr[l].resize(nbox_at(l));
    for (size_t b = 0; b < geo[l].size(); ++b) {
      if (l == 1) {
        const int i = (int)(b / 6), s = (int)(b % 6);
        geo[l][b] = TriBox{{C[i], double2{C[i].x + r0 * std::cos(s * M_PI / 3), C[i].y + r0 * std::sin(s * M_PI / 3)},
                            double2{C[i].x + r0 * std::cos((s + 1) * M_PI / 3),
                                    C[i].y + r0 * std::sin((s + 1) * M_PI / 3)}}};
      } else {
        geo[l][b] = tri_child(geo[l - 1][b >> 2], (int)(b & 3));
      }
      ctr[l][b] = tri_centroid(geo[l][b]);
    }
  }
  const int pmin = h->opt.p_min > 0 ? h->opt.p_min : 30;
  for (int l = 0; l <= D; ++l) {
    Level& L = h->lev[l];
    L.nbox = (int)nbox_at(l);
    const double rl = l == 0 ? r0 : r0 / (s3 * (double)(1 << (l - 1)));   // circumradius
    L.d = 2 * rl;
    std::vector<int> cnt(L.nbox, 0);
    for (int e = 0; e < E; ++e) cnt[key_at(e, l)]++;
    L.hbegin.resize(L.nbox);
    L.hend.resize(L.nbox);
    int acc = 0;
    for (int b = 0; b < L.nbox; ++b) {
      L.hbegin[b] = acc;
      acc += cnt[b];
      L.hend[b] = acc;
      if (cnt[b] > 0) L.hne.push_back(b);
    }
    L.nne = (int)L.hne.size();
    // the square tree's order rule on the cell's diameter; p_min 30 for the
    // triangle tree's larger convergence factor (Table 1: tau 0.6663 against 0.6009)
    const double x = 2 * k * rl;
    int p = h->opt.p > 0 ? h->opt.p : (int)std::ceil(x + 1.8 * std::pow(10.0, 2.0 / 3.0) * std::cbrt(x));
    p = std::max(p, h->opt.p > 0 ? 1 : pmin);
    if (p > PF_PMAX) return fail(h, PFMBEM_EINVAL, "expansion order above the library limit (128); use more levels");
    L.p = L.p32 = p;
    L.P = 2 * p + 1;
    L.sigma = k * rl;
    L.w.assign(L.P, 1.0);
    double wn = 1.0;
    for (int n = 1; n <= p; ++n) {
      wn *= L.sigma / n;
      L.w[p + n] = L.w[p - n] = wn;
    }
    h->info.p[l] = p;
    h->info.p32[l] = p;
  }
  // ---------------------------------------------------- neighbours, M2L lists, near lists
  // level 0: cells whose lattice points are one spacing apart (or the same), images |m| <= 1
  std::vector<std::vector<std::pair<int, int>>> nb_prev(M);
  std::vector<unsigned char> nbr((size_t)M * M * 3, 0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j)
      for (int m = -1; m <= 1; ++m) {
        const double dx = C[i].x - C[j].x, dy = C[i].y - C[j].y - m * H;
        if (std::sqrt(dx * dx + dy * dy) <= a * (1 + 1e-6)) {
          nb_prev[i].push_back({j, m});
          nbr[((size_t)i * M + j) * 3 + m + 1] = 1;
        }
      }
  int64_t m2l_pairs = 0;
  std::vector<OffsetTable> m2l_off(D + 1);
  std::vector<int> nl_ptr(1, 0), nl_src, nl_img;
  for (int l = 1; l <= D; ++l) {
    Level& L = h->lev[l];
    const Level& Lp = h->lev[l - 1];
    const int nch = l == 1 ? 6 : 4;
    const double side = l == 1 ? r0 : r0 / (double)(1 << (l - 1));
    const double tol = 1e-6 * side;
    m2l_off[l].quantum = 1e-7 * side;
    std::vector<std::vector<std::pair<int, int>>> nb(L.nbox);
    std::vector<int> ptr(1, 0), src, off, img, tgt;
    for (int b : L.hne) {
      const int par = b / nch;
      for (const auto& pm : nb_prev[par]) {
        const int B = pm.first, m = pm.second;
        if (Lp.hend[B] <= Lp.hbegin[B]) continue;
        for (int q = 0; q < nch; ++q) {
          const int cb = nch * B + q;
          if (L.hend[cb] <= L.hbegin[cb]) continue;
          if (tri_touch(geo[l][b], geo[l][cb], m * H, tol)) {
            nb[b].push_back({cb, m});
          } else {
            src.push_back(cb);
            img.push_back(m);
            tgt.push_back(b);
            off.push_back(m2l_off[l].get(double2{ctr[l][b].x - ctr[l][cb].x, ctr[l][b].y - ctr[l][cb].y - m * H}));
          }
        }
      }
      ptr.push_back((int)src.size());
      if (l == D) {
        for (const auto& pm : nb[b]) {
          nl_src.push_back(pm.first);
          nl_img.push_back(pm.second);
        }
        nl_ptr.push_back((int)nl_src.size());
      }
    }
    L.nil = (int64_t)src.size();
    m2l_pairs += L.nil;
    h->info.m2l_pairs_level[l] = L.nil;
    pfmbem_status st;
    if ((st = upload(h, &L.il_ptr, ptr)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_src, src)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_off, off)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_img, img)) != PFMBEM_OK) return st;
    {
      // the same pairs grouped by offset, in chunks of at most 16 pairs (the
      // cached product stages one operator per chunk)
      std::vector<int> order(src.size());
      for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return off[x] < off[y]; });
      std::vector<int> ptg, psr, pim, cof, cbg, cen;
      for (size_t i = 0; i < order.size(); ++i) {
        const int q = order[i];
        if (cof.empty() || cof.back() != off[q] || (int)ptg.size() - cbg.back() >= 16) {
          if (!cof.empty()) cen.push_back((int)ptg.size());
          cof.push_back(off[q]);
          cbg.push_back((int)ptg.size());
        }
        ptg.push_back(tgt[q]);
        psr.push_back(src[q]);
        pim.push_back(img[q]);
      }
      if (!cof.empty()) cen.push_back((int)ptg.size());
      L.nchunk = (int)cof.size();
      if ((st = upload(h, &L.pr_tgt, ptg)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.pr_src, psr)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.pr_img, pim)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.ch_off, cof)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.ch_beg, cbg)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.ch_end, cen)) != PFMBEM_OK) return st;
    }
    nb_prev.swap(nb);
  }
  h->info.m2l_pairs = m2l_pairs;
  {
    pfmbem_status st;
    if ((st = upload(h, &h->nl_ptr, nl_ptr)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->nl_src, nl_src)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->nl_img, nl_img)) != PFMBEM_OK) return st;
  }
  // ---------------------------------------------------- cached element integrals
  // As the square tree's: per leaf its concatenated near sources and a dense
  // [targets][sources] array of 2x2 blocks; the same-fiber blocks (a row pair
  // for a regular polygon, whose block is circulant); P2M/L2P coefficients.
  // Without room (or with near_mode 1) the product integrates them every time.
  std::vector<int64_t> nc_base, fbase(M, 0), kbase(M, -1);
  std::vector<int> nc_sbase(1, 0), chunks, circ(M, 0), rows;
  int64_t fb_acc = 0, kacc = 0;
  {
    const Level& Lf = h->lev[D];
    int64_t acc = 0;
    for (size_t li = 0; li < Lf.hne.size(); ++li) {
      const int b = Lf.hne[li];
      int ns = 0;
      for (int e = nl_ptr[li]; e < nl_ptr[li + 1]; ++e) ns += Lf.hend[nl_src[e]] - Lf.hbegin[nl_src[e]];
      nc_sbase.push_back(nc_sbase.back() + ns);
      h->nc_maxns = std::max(h->nc_maxns, ns);
      h->leaf_maxn = std::max(h->leaf_maxn, Lf.hend[b] - Lf.hbegin[b]);
      nc_base.push_back(acc);
      acc += 4 * (int64_t)(Lf.hend[b] - Lf.hbegin[b]) * ns;
    }
    h->nc_blocks = acc / 4;
    for (int i = 0; i < M; ++i) {
      const int n = foff[i + 1] - foff[i], n2 = 2 * n;
      circ[i] = regular_polygon(len, t, foff[i], n) ? 1 : 0;
      fbase[i] = fb_acc;
      fb_acc += circ[i] ? (int64_t)2 * n2 : (int64_t)n2 * n2;
      for (int r = 0; r < n2; r += 32) {
        chunks.push_back(i);
        chunks.push_back(r);
        chunks.push_back(std::min(r + 32, n2));
      }
      for (int e = foff[i]; e < (circ[i] ? foff[i] + 1 : foff[i + 1]); ++e) rows.push_back(e);
      if (circ[i]) {
        kbase[i] = kacc;
        kacc += n;
      }
    }
  }
  {
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    const double bytes = (double)(4 * h->nc_blocks + fb_acc) * (sizeof(cplx) + 2 * sizeof(cplxf)) +
                         2.0 * E * 2 * h->lev[D].P * sizeof(cplx);
    // (the near-field build's shared memory: per-source and per-target arrays)
    const size_t nb_smem = sizeof(int) * (13 * (size_t)h->nc_maxns + 4 * (size_t)h->leaf_maxn + 16);
    h->tri_cache = h->opt.near_mode == 0 && h->max_fiber <= 1024 && bytes < 0.5 * (double)freeb &&
                   nb_smem <= 200 * 1024;
  }
  if (h->tri_cache) {
    h->fb_entries = fb_acc;
    h->hcirc = circ;
    h->nfb_rows = (int)rows.size();
    h->nchunk = (int)chunks.size() / 3;
    pfmbem_status st;
    if ((st = upload(h, &h->nc_base, nc_base)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->nc_sbase, nc_sbase)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fb_base, fbase)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fb_circ, circ)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fb_chunk, chunks)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fb_rows, rows)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->kt_base, kbase)) != PFMBEM_OK) return st;
    if ((st = build_pair_tables(h, nodes, foff, fib, std::vector<int>(E, 0), perm, nl_ptr, nl_src, nl_img)) !=
        PFMBEM_OK)
      return st;
    h->nc_src = dalloc<int>(h, (size_t)std::max(nc_sbase.back(), 1));
    h->nc_img = dalloc<int>(h, (size_t)std::max(nc_sbase.back(), 1));
    h->kt_val = dalloc<cplx>(h, (size_t)4 * kacc);
    h->kt_sval = dalloc<cplx>(h, (size_t)4 * kacc);
    h->kt_svalf = dalloc<cplxf>(h, (size_t)4 * kacc);
    h->kt_svall = dalloc<cplxf>(h, (size_t)4 * kacc);
    h->nq_cap = (unsigned)std::min<int64_t>(h->nc_blocks, (int64_t)0xFFFFFFFFu);
    h->nq = dalloc<unsigned long long>(h, std::max<size_t>(h->nq_cap, 1));
    h->nq_len = dalloc<unsigned>(h, 1);
    h->nc_valf = dalloc<cplxf>(h, (size_t)(4 * h->nc_blocks));
    h->nc_vall = dalloc<cplxf>(h, (size_t)(4 * h->nc_blocks));
    h->fb_val = dalloc<cplx>(h, (size_t)fb_acc);
    h->fb_valf = dalloc<cplxf>(h, (size_t)fb_acc);
    h->stat_dev = dalloc<unsigned long long>(h, 4);
    const size_t ncoef = (size_t)E * 2 * h->lev[D].P;
    h->p2m_c = dalloc<cplx>(h, ncoef);
    h->l2p_c = dalloc<cplx>(h, ncoef);
    if (!h->nc_src || !h->nc_img || !h->kt_val || !h->kt_sval || !h->kt_svalf || !h->kt_svall || !h->nq ||
        !h->nq_len || !h->nc_valf || !h->nc_vall || !h->fb_val || !h->fb_valf || !h->stat_dev || !h->p2m_c ||
        !h->l2p_c)
      return fail(h, PFMBEM_ENOMEM, "device allocation failed (triangle tree caches)");
    CK(cudaMemsetAsync(h->stat_dev, 0, 4 * sizeof(unsigned long long), h->stream));
  }
  // near-field and same-fiber pair statistics on the host when the product
  // integrates them every time (the cache build counts them on the GPU)
  if (!h->tri_cache) {
    const Level& Lf = h->lev[D];
    int64_t pairs = 0, quad = 0;
    for (size_t li = 0; li < Lf.hne.size(); ++li) {
      const int b = Lf.hne[li];
      for (int s = Lf.hbegin[b]; s < Lf.hend[b]; ++s)
        for (int e = nl_ptr[li]; e < nl_ptr[li + 1]; ++e)
          for (int f = Lf.hbegin[nl_src[e]]; f < Lf.hend[nl_src[e]]; ++f) {
            if (f == s && nl_img[e] == 0) continue;
            const int eo = perm[f], so = perm[s];
            const double q = std::hypot(c[so].x - c[eo].x, c[so].y - (c[eo].y + nl_img[e] * H)) / len[eo];
            pairs++;
            quad += gl_order_host(q, g_thr64);
          }
    }
    h->info.near_pairs = pairs;
    h->info.near_quad = quad;
    pairs = quad = 0;
    for (int i = 0; i < M; ++i)
      for (int e = foff[i]; e < foff[i + 1]; ++e)
        for (int f = foff[i]; f < foff[i + 1]; ++f) {
          if (f == e) continue;
          pairs++;
          quad += gl_order_host(std::hypot(c[e].x - c[f].x, c[e].y - c[f].y) / len[f], g_thr64);
        }
    h->info.fiber_pairs = pairs;
    h->info.fiber_quad = quad;
  }
  // P2M Gauss nodes: a leaf's M2L sources are at least the leaf triangle's height
  // (side sqrt(3) / 2) away
  {
    const double sideD = D == 1 ? r0 : r0 / (double)(1 << (D - 1));
    const double qfar = std::max(1.0, 0.5 * s3 * sideD / hmax - 1.0);
    h->g_far = gl_order_host(qfar, g_thr64);
    h->g_far_f = gl_order_host(qfar, g_thr32);
  }
  // ---------------------------------------------------- M2M / L2L offsets (child - parent)
  std::vector<OffsetTable> sh_off(D);
  for (int l = 0; l < D; ++l) {
    Level& Lc = h->lev[l + 1];
    const int nch = l == 0 ? 6 : 4;
    sh_off[l].quantum = 1e-7 * (l == 0 ? r0 : r0 / (double)(1 << l));
    std::vector<int> pidx(Lc.nbox, 0);
    for (int b = 0; b < Lc.nbox; ++b) {
      const int par = b / nch;
      pidx[b] = sh_off[l].get(double2{ctr[l + 1][b].x - ctr[l][par].x, ctr[l + 1][b].y - ctr[l][par].y});
    }
    pfmbem_status st;
    if ((st = upload(h, &Lc.pidx, pidx)) != PFMBEM_OK) return st;
  }
  // ---------------------------------------------------- level arrays
  std::vector<double2*> m2l_v(D + 1, nullptr), sh_v(D + 1, nullptr);
  for (int l = 0; l <= D; ++l) {
    Level& L = h->lev[l];
    pfmbem_status st;
    if ((st = upload(h, &L.w_dev, L.w)) != PFMBEM_OK) return st;
    {
      std::vector<double> iw(L.w.size());
      for (size_t i = 0; i < iw.size(); ++i) iw[i] = 1.0 / L.w[i];
      if ((st = upload(h, &L.iw_dev, iw)) != PFMBEM_OK) return st;
    }
    if ((st = upload(h, &L.ne, L.hne)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.box_begin, L.hbegin)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.box_end, L.hend)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.ctr, ctr[l])) != PFMBEM_OK) return st;
    if (l >= 1 && !m2l_off[l].v.empty() && (st = upload(h, &m2l_v[l], m2l_off[l].v)) != PFMBEM_OK) return st;
    if (l < D && (st = upload(h, &sh_v[l], sh_off[l].v)) != PFMBEM_OK) return st;
    L.M = dalloc<cplx>(h, (size_t)L.nbox * L.P);
    L.L = dalloc<cplx>(h, (size_t)L.nbox * L.P);
    if (!L.M || !L.L) return fail(h, PFMBEM_ENOMEM, "device allocation failed (expansions)");
    if (l >= 1) {
      L.tri_noff = (int)m2l_off[l].v.size();
      L.m2l = dalloc<cplx>(h, std::max<size_t>(m2l_off[l].v.size(), 1) * L.P * L.P);
      if (!L.m2l) return fail(h, PFMBEM_ENOMEM, "device allocation failed (M2L operators)");
      if (h->tri_cache && L.tri_noff > 0) {
        // hi and lo parts for the double-float M2L of the cached product
        L.tri_m2l_hl = dalloc<cplxf>(h, 2 * (size_t)L.tri_noff * L.P * L.P);
        if (!L.tri_m2l_hl) return fail(h, PFMBEM_ENOMEM, "device allocation failed (M2L operators)");
      }
    }
    if (l < D) {
      L.tri_nop = (int)sh_off[l].v.size();
      const size_t n = sh_off[l].v.size() * L.P * h->lev[l + 1].P;
      L.m2m = dalloc<cplx>(h, n);
      L.l2l = dalloc<cplx>(h, n);
      if (!L.m2m || !L.l2l) return fail(h, PFMBEM_ENOMEM, "device allocation failed (M2M/L2L operators)");
      if (h->tri_cache) {
        // hi and lo parts for the double-float M2M and L2L of the cached product
        L.tri_m2m_hl = dalloc<cplxf>(h, 2 * n);
        L.tri_l2l_hl = dalloc<cplxf>(h, 2 * n);
        if (!L.tri_m2m_hl || !L.tri_l2l_hl) return fail(h, PFMBEM_ENOMEM, "device allocation failed (M2M/L2L operators)");
      }
    }
  }
  // ---------------------------------------------------- element arrays (no wrapping: m0 = 0)
  {
    std::vector<int> m0(E, 0);
    pfmbem_status st;
    if ((st = upload(h, &h->s_perm, perm)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_m0, m0)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_key, key)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_c, c)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_t, t)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_nu, nu)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_h, len)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_fiber, fib)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fib_off, foff)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->fib_geo, h->hfib_geo)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->o_pos, pos)) != PFMBEM_OK) return st;
  }
  h->s_c = dalloc<double2>(h, (size_t)E);
  h->s_t = dalloc<double2>(h, (size_t)E);
  h->s_nu = dalloc<double2>(h, (size_t)E);
  h->s_h = dalloc<double>(h, (size_t)E);
  h->s_ph = dalloc<cplx>(h, (size_t)E);
  h->s_m0 = dalloc<int>(h, (size_t)E);
  h->s_leaf = dalloc<int>(h, (size_t)E);
  h->self4 = dalloc<cplx>(h, (size_t)4 * E);
  h->dens = dalloc<cplx>(h, (size_t)2 * E);
  h->U = dalloc<cplx>(h, (size_t)2 * E);
  h->stage_in = dalloc<cplx>(h, (size_t)2 * E);
  h->stage_out = dalloc<cplx>(h, (size_t)2 * E);
  h->dev_rhs = dalloc<cplx>(h, (size_t)2 * E);
  h->tab_err = dalloc<int>(h, 1);
  if (!h->s_c || !h->s_t || !h->s_nu || !h->s_h || !h->s_ph || !h->s_m0 || !h->s_leaf || !h->self4 || !h->dens ||
      !h->U || !h->stage_in || !h->stage_out || !h->dev_rhs || !h->tab_err)
    return fail(h, PFMBEM_ENOMEM, "device allocation failed (element arrays)");
  // ---------------------------------------------------- the operator between the cells
  // super root: centre of the cells' bounding box, radius over the cells'
  // circles; images |m| >= m0 (m0 H >= 3 R_s, at least 2) through its lattice sums
  double xmn = 1e300, xmx = -1e300, ymn = 1e300, ymx = -1e300;
  for (int i = 0; i < M; ++i) {
    xmn = std::min(xmn, C[i].x - r0); xmx = std::max(xmx, C[i].x + r0);
    ymn = std::min(ymn, C[i].y - r0); ymx = std::max(ymx, C[i].y + r0);
  }
  h->nroot = M;
  h->wide_cx = 0.5 * (xmn + xmx);
  h->wide_cy = 0.5 * (ymn + ymx);
  h->wide_rs = 0;
  for (int i = 0; i < M; ++i)
    h->wide_rs = std::max(h->wide_rs, std::hypot(C[i].x - h->wide_cx, C[i].y - h->wide_cy) + r0);
  h->wide_m0 = std::max(2, (int)std::ceil(3.0 * h->wide_rs / H - 1e-12));
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j)
      for (int m = -(h->wide_m0 - 1); m <= h->wide_m0 - 1; ++m) {
        if (std::abs(m) <= 1) continue;
        if (std::hypot(C[i].x - C[j].x, C[i].y - C[j].y - m * H) <= a * (1 + 1e-6))
          return fail(h, PFMBEM_EGEOM, "triangle tree: cells touch across two periods (block taller than H)");
      }
  {
    const double x = 2.0 * k * h->wide_rs;
    const int pratio = (int)std::ceil(std::log(1e-11) / std::log(2.0 * h->wide_rs / (h->wide_m0 * H)));
    const int ps = std::max({(int)std::ceil(x + 1.8 * std::pow(10.0, 2.0 / 3.0) * std::cbrt(x)), h->lev[0].p, pratio});
    if (ps > PF_PMAX) return fail(h, PFMBEM_EINVAL, "block too large for this frequency (super-root order above 128)");
    h->wide_ps = ps;
  }
  h->x0 = xmn;
  h->y0 = h->wide_cy - 0.5 * H;
  h->field_hw = 0.5 * (xmx - xmn);
  const int P0 = h->lev[0].P, ps = h->wide_ps, Ps = 2 * ps + 1;
  if ((double)M * P0 * M * P0 * sizeof(cplx) > 8e9)
    return fail(h, PFMBEM_EINVAL, "triangle tree: too many cells for the dense operator between them");
  unsigned char* nbr_dev = nullptr;
  double2* dv = nullptr;
  {
    std::vector<double2> hv(2 * (size_t)M);
    for (int i = 0; i < M; ++i) {
      hv[i] = C[i];
      hv[M + i] = double2{C[i].x - h->wide_cx, C[i].y - h->wide_cy};
    }
    std::vector<double> w(Ps, 1.0);
    double wn = 1.0;
    for (int n = 1; n <= ps; ++n) {
      wn *= k * h->wide_rs / n;
      w[ps + n] = w[ps - n] = wn;
    }
    pfmbem_status st;
    if ((st = upload(h, &dv, hv)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->wide_w, w)) != PFMBEM_OK) return st;
    if ((st = upload(h, &nbr_dev, nbr)) != PFMBEM_OK) return st;
    if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
  }
  h->root = dalloc<cplx>(h, (size_t)M * P0 * M * P0);
  h->wide_A = dalloc<cplx>(h, (size_t)M * P0 * Ps);
  h->wide_B = dalloc<cplx>(h, (size_t)M * Ps * P0);
  h->wide_Rs = dalloc<cplx>(h, (size_t)Ps * Ps);
  h->wide_ML = dalloc<cplx>(h, 2 * (size_t)Ps);
  cplx* S = dalloc<cplx>(h, (size_t)2 * ps + 1);
  cplx* X = dalloc<cplx>(h, (size_t)M * Ps * P0);
  if (!h->root || !h->wide_A || !h->wide_B || !h->wide_Rs || !h->wide_ML || !S || !X)
    return fail(h, PFMBEM_ENOMEM, "device allocation failed (operator between the cells)");
  CK(cudaMemsetAsync(h->tab_err, 0, sizeof(int), h->stream));
  CK(k_sort_elements(h));
  CK(k_self_terms(h));
  for (int l = 0; l <= D; ++l)
    CK(k_tri_tables(h, l, l >= 1 ? m2l_v[l] : nullptr, l >= 1 ? (int)m2l_off[l].v.size() : 0,
                    l < D ? sh_v[l] : nullptr, l < D ? (int)sh_off[l].v.size() : 0));
  CK(k_wide_top(h, dv, S, X, nbr_dev));
  if (h->tri_cache) {
    CK(k_tri_caches(h));
    for (int l = 0; l <= D; ++l) CK(k_tri_m2l_split(h, l));
  }
  h->ub_on = false;
  pin_release_async(h);
  h->info.E = E;
  h->info.M = M;
  h->info.depth = D;
  h->info.nleaf_nonempty = h->lev[D].nne;
  h->info.p2m_nodes = h->g_far;
  h->info.lattice_q = h->lattice_q;
  h->info.root_x0 = h->x0;
  h->info.root_y0 = h->y0;
  h->info.nroot = M;
  h->info.super_p = ps;
  h->setup_ms = now_ms() - t0;
  h->info.setup_ms = h->setup_ms;
  return PFMBEM_OK;
}
