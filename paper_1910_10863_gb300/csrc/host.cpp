// Host side of the pfmbem library: geometry checks, the periodic quadtree
// (Sec. 3.1), translation tables (Sec. 3.2), the lattice-sum root operator
// (Sec. 3.3), the C ABI and the GMRES driver (Sec. 4).
#include <algorithm>
#include <chrono>
#include <complex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <future>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

pfmbem_status fail(pfmbem* h, pfmbem_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

pfmbem_status fail_cuda(pfmbem* h, cudaError_t e, const char* what) {
  if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PFMBEM_ENOMEM : PFMBEM_ECUDA;
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return fail_cuda(h, _e, #call);  \
  } while (0)

// Device allocations come from the device's stream-ordered memory pool, which
// keeps released memory for reuse (release threshold raised once per device),
// so that repeated create/destroy cycles of a sweep do not map memory again.
void ensure_pool() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

// Small arrays are carved from per-stream chunks of the handle, so that a
// create makes a handful of pool allocations instead of about a hundred: the
// pool's allocation call slows down by an order of magnitude once many
// handles have come and gone (its free lists grow), and every create and solve
// paid for each call.  A carve is ordered on the stream its chunk was
// allocated on, as the allocation itself was; chunks and the arrays too large
// to carve are released together at destroy.
constexpr size_t kCarveMax = (size_t)256 << 10;     // largest carved array
constexpr size_t kChunkMin = (size_t)512 << 10;
constexpr size_t kChunkMax = (size_t)8 << 20;

void* dalloc_bytes(pfmbem* h, size_t bytes, bool carve) {
  cudaStream_t st = h->astream ? h->astream : h->stream;
  bytes = (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
  if (carve && bytes <= kCarveMax) {
    pfmbem::Carve* c = nullptr;
    for (auto& x : h->carves)
      if (x.stream == st) c = &x;
    if (c && c->used + bytes <= c->cap) {
      void* p = c->base + c->used;
      c->used += bytes;
      return p;
    }
    const size_t cap = std::min(kChunkMax, std::max(kChunkMin, c ? 2 * c->cap : kChunkMin));
    void* base = nullptr;
    if (cudaMallocAsync(&base, cap, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    h->allocs.push_back(base);
    if (!c) {
      h->carves.push_back({});
      c = &h->carves.back();
      c->stream = st;
    }
    c->base = static_cast<unsigned char*>(base);
    c->cap = cap;
    c->used = bytes;
    return base;
  }
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  h->allocs.push_back(p);
  return p;
}

template <class T>
T* dalloc(pfmbem* h, size_t n) {
  return static_cast<T*>(dalloc_bytes(h, n * sizeof(T), true));
}

// A temporary released on its own before destroy (never carved).
template <class T>
T* dalloc_tmp(pfmbem* h, size_t n) {
  return static_cast<T*>(dalloc_bytes(h, n * sizeof(T), false));
}

// Page-locked staging for the batched set-up copies: one process-wide arena,
// held by one create at a time (pin_acquire to pin_release).  A create that
// ends without waiting for its stream lets go with pin_release_async, which
// records an event after its last copy; the next holder waits for that event
// before it writes into the arena.  A create that finds the arena held by
// another, or whose batches outgrow it, stages in pageable memory.
struct PinnedArena {
  std::mutex mu;
  unsigned char* buf = nullptr;
  size_t cap = 0;
  pfmbem* owner = nullptr;
  cudaEvent_t done = nullptr;      // after the last copy of the previous holder
  int done_dev = -1;
  bool pending = false;
};
PinnedArena g_pin;

void pin_acquire(pfmbem* h) {
  std::lock_guard<std::mutex> lk(g_pin.mu);
  h->pin_user = true;
  if (!g_pin.buf) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, (size_t)64 << 20, cudaHostAllocDefault) == cudaSuccess) {
      g_pin.buf = static_cast<unsigned char*>(p);
      g_pin.cap = (size_t)64 << 20;
    } else {
      cudaGetLastError();
    }
  }
  if (g_pin.buf && !g_pin.owner) {
    if (g_pin.pending) {
      cudaEventSynchronize(g_pin.done);
      cudaGetLastError();
      g_pin.pending = false;
    }
    g_pin.owner = h;
    h->ub_pin = g_pin.buf;
    h->ub_pin_cap = g_pin.cap;
    h->ub_pin_batch = 0;
    h->ub_len = 0;
  }
}

void pin_release(pfmbem* h) {
  if (!h->pin_user) return;
  std::lock_guard<std::mutex> lk(g_pin.mu);
  if (g_pin.owner == h) g_pin.owner = nullptr;
  h->ub_pin = nullptr;
  h->pin_user = false;
}

// Lets go of the arena without waiting: the next holder waits for the event
// recorded here (or, on another device, this create waits now).
void pin_release_async(pfmbem* h) {
  if (!h->pin_user) return;
  std::lock_guard<std::mutex> lk(g_pin.mu);
  if (g_pin.owner == h) {
    bool queued = false;
    if (!g_pin.done && cudaEventCreateWithFlags(&g_pin.done, cudaEventDisableTiming) == cudaSuccess)
      g_pin.done_dev = h->dev;
    if (g_pin.done && g_pin.done_dev == h->dev && cudaEventRecord(g_pin.done, h->stream) == cudaSuccess)
      queued = true;
    cudaGetLastError();
    if (!queued) cudaStreamSynchronize(h->stream);
    g_pin.pending = queued;
    g_pin.owner = nullptr;
  }
  h->ub_pin = nullptr;
  h->pin_user = false;
}

// Set-up streams and events are kept in a process-wide pool per device and
// handed from one create to the next: creating and destroying them costs more
// than a small create's host work.  A handle holds its streams exclusively
// between create and destroy; destroy synchronises them before it returns them.
struct StreamPool {
  std::mutex mu;
  std::vector<cudaStream_t> streams[64], hstreams[64];   // default / highest priority
  std::vector<cudaEvent_t> events[64];
};
StreamPool g_sp;

cudaError_t pool_stream(int dev, cudaStream_t* s, bool hi = false) {
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_sp.mu);
    auto& v = hi ? g_sp.hstreams[dev] : g_sp.streams[dev];
    if (!v.empty()) {
      *s = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  if (hi) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, greatest);
  }
  return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}

cudaError_t pool_event(int dev, cudaEvent_t* e) {
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_sp.mu);
    if (!g_sp.events[dev].empty()) {
      *e = g_sp.events[dev].back();
      g_sp.events[dev].pop_back();
      return cudaSuccess;
    }
  }
  return cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

void pool_put(int dev, cudaStream_t s, bool hi = false) {
  if (!s) return;
  if (dev < 0 || dev >= 64) {
    cudaStreamDestroy(s);
    return;
  }
  std::lock_guard<std::mutex> lk(g_sp.mu);
  (hi ? g_sp.hstreams[dev] : g_sp.streams[dev]).push_back(s);
}

void pool_put(int dev, cudaEvent_t e) {
  if (!e) return;
  if (dev < 0 || dev >= 64) {
    cudaEventDestroy(e);
    return;
  }
  std::lock_guard<std::mutex> lk(g_sp.mu);
  g_sp.events[dev].push_back(e);
}

// Host-to-device copy of a table.  While a batch is open (h->ub_on) the data is
// appended to the batch (in the page-locked arena when this create holds it)
// and the destination pointer is set at the next flush_uploads, which makes
// one allocation and one copy for the whole batch.
template <class T>
pfmbem_status upload(pfmbem* h, T** dst, const std::vector<T>& src) {
  const size_t nb = src.size() * sizeof(T);
  if (h->ub_on) {
    if (h->ub_pin && !h->ub_spill) {
      const size_t off = (h->ub_len + 255) & ~(size_t)255;
      if (h->ub_pin_batch + off + nb <= h->ub_pin_cap) {
        if (nb) std::memcpy(h->ub_pin + h->ub_pin_batch + off, src.data(), nb);
        h->ub_len = off + nb;
        h->ub_fix.push_back({reinterpret_cast<void**>(dst), off});
        *dst = nullptr;
        return PFMBEM_OK;
      }
      // the arena is full: the open batch continues in pageable memory
      h->ub_buf.resize(h->ub_len);
      if (h->ub_len) std::memcpy(h->ub_buf.data(), h->ub_pin + h->ub_pin_batch, h->ub_len);
      h->ub_len = 0;
      h->ub_spill = true;
    }
    const size_t off = (h->ub_buf.size() + 255) & ~(size_t)255;
    h->ub_buf.resize(off + nb);
    if (nb) std::memcpy(h->ub_buf.data() + off, src.data(), nb);
    h->ub_fix.push_back({reinterpret_cast<void**>(dst), off});
    *dst = nullptr;
    return PFMBEM_OK;
  }
  *dst = dalloc<T>(h, src.size());
  if (!*dst) return fail(h, PFMBEM_ENOMEM, "device allocation failed");
  if (nb) CK(cudaMemcpyAsync(*dst, src.data(), nb, cudaMemcpyHostToDevice, h->astream ? h->astream : h->stream));
  return PFMBEM_OK;
}

// Copies the open batch to the device and sets its destination pointers; the
// batch stays open.
pfmbem_status flush_uploads(pfmbem* h) {
  if (h->ub_fix.empty()) return PFMBEM_OK;
  cudaStream_t st = h->astream ? h->astream : h->stream;
  const bool pinned = h->ub_pin && !h->ub_spill;
  const size_t nb = pinned ? h->ub_len : h->ub_buf.size();
  unsigned char* d = dalloc<unsigned char>(h, std::max<size_t>(nb, 1));
  if (!d) return fail(h, PFMBEM_ENOMEM, "device allocation failed");
  if (nb) CK(cudaMemcpyAsync(d, pinned ? h->ub_pin + h->ub_pin_batch : h->ub_buf.data(), nb, cudaMemcpyHostToDevice, st));
  for (auto& f : h->ub_fix) *f.first = d + f.second;
  if (pinned) {
    h->ub_pin_batch += (nb + 255) & ~(size_t)255;   // the copy may still be reading the batch
    h->ub_len = 0;
  }
  h->ub_buf.clear();
  h->ub_fix.clear();
  h->ub_spill = false;
  return PFMBEM_OK;
}

std::vector<cplxf> to_float(const std::vector<cplx>& v) {
  std::vector<cplxf> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = cplxf{(float)v[i].re, (float)v[i].im};
  return o;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void trace(pfmbem* h, cudaStream_t st, const char* label) {
  if (!h->trace_on) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess || cudaEventRecord(e, st) != cudaSuccess) {
    cudaGetLastError();
    if (e) cudaEventDestroy(e);
    return;
  }
  h->trace_lbl.push_back(label);
  h->trace_ev.push_back(e);
  h->trace_host.push_back(now_ms());
}

namespace {

// Prints the set-up trace (GPU time of each event and host time of its record,
// both from the first) once the streams have completed, and releases it.
static void trace_report(pfmbem* h) {
  if (h->trace_ev.empty()) return;
  for (size_t i = 0; i < h->trace_ev.size(); ++i) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->trace_ev[0], h->trace_ev[i]);
    std::fprintf(stderr, "pfmbem trace %-34s gpu %7.3f ms  host %7.3f ms\n", h->trace_lbl[i], ms,
                 h->trace_host[i] - h->trace_host[0]);
  }
  for (cudaEvent_t e : h->trace_ev) cudaEventDestroy(e);
  h->trace_ev.clear();
  h->trace_lbl.clear();
  h->trace_host.clear();
}

// Spreads the low 16 bits of v to the even bit positions.
inline unsigned spread_bits(unsigned v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Gathers the even bit positions of v (inverse of spread_bits).
inline unsigned unspread_bits(unsigned v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}

// Morton code of box (ix, iy) at depth D: bit b of ix to bit 2b, of iy to 2b + 1.
inline int morton(int ix, int iy, int D) {
  const unsigned m = (1u << D) - 1u;
  return (int)(spread_bits((unsigned)ix & m) | (spread_bits((unsigned)iy & m) << 1));
}

// Root squares of side H along x (at most kMaxRoots): box (ix, iy) of level l,
// ix < nroot 2^l, is numbered root-major, root (ix >> l) first and the Morton code
// inside it after, so that a box's children are 4 b .. 4 b + 3 and its parent b >> 2
// as in one root, and the level's boxes of one root are consecutive.
constexpr int kMaxRoots = 4;
inline int box_id(int ix, int iy, int l) { return ((ix >> l) << (2 * l)) | morton(ix & ((1 << l) - 1), iy, l); }
inline void box_xy(int b, int l, int* ix, int* iy) {
  const unsigned m = (unsigned)b & ((1u << (2 * l)) - 1u);
  *ix = ((b >> (2 * l)) << l) | (int)unspread_bits(m);
  *iy = (int)unspread_bits(m >> 1);
}

// Gauss-Legendre thresholds: rule g meets tolerance tol for a source element
// whose midpoint is q element lengths away when its Bernstein ellipse
// parameter 2q + sqrt(4q^2 - 1) >= tol^(-1/(2g)); i.e. q >= (R + 1/R)/4.
void gl_thresholds(double tol, double* thr) {
  thr[0] = 1e300;
  for (int g = 1; g <= PF_GLMAX; ++g) {
    double R = std::pow(tol, -1.0 / (2.0 * g));
    thr[g] = (R + 1.0 / R) / 4.0;
  }
}

int gl_order_host(double q, const double* thr) {
  int g = 1;
  while (g < PF_GLMAX && q < thr[g]) ++g;
  return g;
}

double g_thr64[PF_GLMAX + 1], g_thr32[PF_GLMAX + 1];
int g_gauss_ready_dev = -1;

void ensure_gauss() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_gauss_ready_dev == dev) return;
  std::vector<double> x(PF_GLMAX * PF_GLMAX, 0.0), w(PF_GLMAX * PF_GLMAX, 0.0);
  for (int g = 1; g <= PF_GLMAX; ++g) gauss_legendre(g, &x[(g - 1) * PF_GLMAX], &w[(g - 1) * PF_GLMAX]);
  gl_thresholds(1e-14, g_thr64);
  gl_thresholds(3e-8, g_thr32);
  k_upload_gauss(x.data(), w.data(), g_thr64, g_thr32);
  k_upload_series();
  g_gauss_ready_dev = dev;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // final derivative at the converged node
        p0 = 1.0; p1 = z;
        for (int j = 2; j <= n; ++j) {
          double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p1 = z; p0 = 1.0; }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ============================================================== planning
// Near-field integrals shared by translated copies of a fiber pair.  Fibers
// whose node lists are translates of each other (to 1e-12 H) form a class; a
// near-field fiber pair (A, B, m: source shifted by m periods) is keyed by the
// classes of A and B and the offset between their first nodes.  Keys met at
// least twice get one table of S, D, K, T over all element pairs, built from
// the first pair with the key; the near-field build reads every pair of such a
// key from it.  Nothing happens unless two fibers are congruent.
static pfmbem_status build_pair_tables(pfmbem* h, const double* nodes, const std::vector<int>& foff,
                                       const std::vector<int>& fib, const std::vector<int>& m0,
                                       const std::vector<int>& perm, const std::vector<int>& nl_ptr,
                                       const std::vector<int>& nl_src, const std::vector<int>& nl_img) {
  const int M = h->M, D = h->D;
  const double H = h->H, tol = 1e-12 * H;
  // ---- classes
  std::vector<int> cls(M, -1);
  std::vector<int> rep;                                   // first fiber of each class
  std::map<std::vector<long long>, std::vector<int>> bucket;
  const double q = 1e-9 * H;
  bool repeat = false;
  for (int i = 0; i < M; ++i) {
    const int n = foff[i + 1] - foff[i];
    const double* a = nodes + 2 * foff[i];
    std::vector<long long> key{n};
    for (int j : {1, n / 3, (2 * n) / 3})
      if (j > 0 && j < n) {
        key.push_back(std::llround((a[2 * j] - a[0]) / q));
        key.push_back(std::llround((a[2 * j + 1] - a[1]) / q));
      }
    auto& cand = bucket[key];
    for (int c : cand) {
      const double* r = nodes + 2 * foff[rep[c]];
      bool same = true;
      for (int j = 1; j < n && same; ++j)
        same = std::fabs((a[2 * j] - a[0]) - (r[2 * j] - r[0])) <= tol &&
               std::fabs((a[2 * j + 1] - a[1]) - (r[2 * j + 1] - r[1])) <= tol;
      if (same) {
        cls[i] = c;
        repeat = true;
        break;
      }
    }
    if (cls[i] < 0) {
      cls[i] = (int)rep.size();
      rep.push_back(i);
      cand.push_back(cls[i]);
    }
  }
  if (!repeat) return PFMBEM_OK;
  // ---- near-field fiber pairs (target fiber, source fiber, image shift)
  const Level& Lf = h->lev[D];
  std::vector<unsigned long long> pairs;
  auto pack = [](int A, int B, int m) {
    return ((unsigned long long)(unsigned)A << 32) | ((unsigned long long)(unsigned)B << 8) | (unsigned)(m + 64);
  };
  // distinct (fiber, m0) of every leaf (a leaf's elements of one fiber are
  // contiguous: the sort by leaf key is stable and the input is fiber-major)
  std::vector<int> run_ptr(Lf.nbox + 1, 0);
  std::vector<std::pair<int, int>> runs;
  {
    std::vector<int> first(Lf.nbox, -1), count(Lf.nbox, 0);
    for (int b : Lf.hne) {
      first[b] = (int)runs.size();
      for (int s2 = Lf.hbegin[b]; s2 < Lf.hend[b]; ++s2) {
        const int e = perm[s2];
        const std::pair<int, int> v{fib[e], m0[e]};
        bool seen = false;
        for (int r = first[b]; r < (int)runs.size() && !seen; ++r) seen = runs[r] == v;
        if (!seen) runs.push_back(v);
      }
      count[b] = (int)runs.size() - first[b];
    }
    for (int b = 0; b < Lf.nbox; ++b) run_ptr[b + 1] = run_ptr[b] + (first[b] >= 0 ? count[b] : 0);
    std::vector<std::pair<int, int>> ordered;
    ordered.reserve(runs.size());
    for (int b = 0; b < Lf.nbox; ++b)
      if (first[b] >= 0) ordered.insert(ordered.end(), runs.begin() + first[b], runs.begin() + first[b] + count[b]);
    runs.swap(ordered);
  }
  std::vector<std::pair<int, int>> T;                     // (fiber, m0) of the leaf's targets
  std::vector<std::array<int, 3>> S;                      // (fiber, m0, m) of its sources
  for (size_t li = 0; li < Lf.hne.size(); ++li) {
    const int b = Lf.hne[li];
    T.assign(runs.begin() + run_ptr[b], runs.begin() + run_ptr[b + 1]);
    S.clear();
    for (int j = nl_ptr[li]; j < nl_ptr[li + 1]; ++j) {
      const int sb = nl_src[j];
      for (int r = run_ptr[sb]; r < run_ptr[sb + 1]; ++r) {
        const std::array<int, 3> v{runs[r].first, runs[r].second, nl_img[j]};
        if (std::find(S.begin(), S.end(), v) == S.end()) S.push_back(v);
      }
    }
    for (auto& t : T)
      for (auto& sv : S) {
        const int mt = sv[2] + t.second - sv[1];
        if (sv[0] == t.first && mt == 0) continue;
        if (mt < -60 || mt > 60) continue;
        pairs.push_back(pack(t.first, sv[0], mt));
      }
  }
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  // ---- keys: classes and the offset between the first nodes
  struct Key {
    int ca, cb;
    long long dx, dy;
    bool operator<(const Key& o) const {
      return std::tie(ca, cb, dx, dy) < std::tie(o.ca, o.cb, o.dx, o.dy);
    }
  };
  std::map<Key, int> kid;
  std::vector<int> kcount, kA, kB, km;
  std::vector<int> pair_key(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) {
    const int A = (int)(pairs[i] >> 32), B = (int)((pairs[i] >> 8) & 0xFFFFFF), mt = (int)(pairs[i] & 0xFF) - 64;
    const double* a = nodes + 2 * foff[A];
    const double* bn = nodes + 2 * foff[B];
    const Key key{cls[A], cls[B], std::llround((bn[0] - a[0]) / q), std::llround((bn[1] + mt * H - a[1]) / q)};
    auto it = kid.find(key);
    int id;
    if (it == kid.end()) {
      id = (int)kcount.size();
      kid.emplace(key, id);
      kcount.push_back(0);
      kA.push_back(A);
      kB.push_back(B);
      km.push_back(mt);
    } else {
      id = it->second;
    }
    kcount[id]++;
    pair_key[i] = id;
  }
  // ---- tables for the keys met at least twice
  std::vector<int> tab_of(kcount.size(), -1), tA, tB, tm, tnb;
  std::vector<int64_t> tstart(1, 0);
  for (size_t id = 0; id < kcount.size(); ++id)
    if (kcount[id] >= 2) {
      tab_of[id] = (int)tA.size();
      tA.push_back(kA[id]);
      tB.push_back(kB[id]);
      tm.push_back(km[id]);
      const int na = foff[kA[id] + 1] - foff[kA[id]], nb = foff[kB[id] + 1] - foff[kB[id]];
      tnb.push_back(nb);
      tstart.push_back(tstart.back() + (int64_t)na * nb);
    }
  if (tA.empty()) return PFMBEM_OK;
  std::vector<int> plp(M + 1, 0), plf, pli, plt;
  for (size_t i = 0; i < pairs.size(); ++i)
    if (tab_of[pair_key[i]] >= 0) plp[(pairs[i] >> 32) + 1]++;
  for (int i = 0; i < M; ++i) plp[i + 1] += plp[i];
  plf.resize(plp[M]);
  pli.resize(plp[M]);
  plt.resize(plp[M]);
  {
    std::vector<int> fill(plp.begin(), plp.end() - 1);
    for (size_t i = 0; i < pairs.size(); ++i) {
      const int t = tab_of[pair_key[i]];
      if (t < 0) continue;
      const int A = (int)(pairs[i] >> 32);
      const int at = fill[A]++;
      plf[at] = (int)((pairs[i] >> 8) & 0xFFFFFF);
      pli[at] = (int)(pairs[i] & 0xFF) - 64;
      plt[at] = t;
    }
  }
  h->ntab = (int)tA.size();
  h->tab_entries = tstart.back();
  pfmbem_status st;
  if ((st = upload(h, &h->tab_A, tA)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->tab_B, tB)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->tab_m, tm)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->tab_nb, tnb)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->tab_start, tstart)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->pl_ptr, plp)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->pl_fib, plf)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->pl_img, pli)) != PFMBEM_OK) return st;
  if ((st = upload(h, &h->pl_tab, plt)) != PFMBEM_OK) return st;
  h->tab_val = dalloc<cplx>(h, (size_t)4 * h->tab_entries);
  h->tab_valf = dalloc<cplxf>(h, (size_t)4 * h->tab_entries);
  h->tab_vall = dalloc<cplxf>(h, (size_t)4 * h->tab_entries);
  if (!h->tab_val || !h->tab_valf || !h->tab_vall)
    return fail(h, PFMBEM_ENOMEM, "device allocation failed (fiber-pair tables)");
  return PFMBEM_OK;
}

// M2L interaction lists of one level (host only, no CUDA calls: it runs on a
// worker thread while the set-up continues).  Per non-empty target box the
// sources are the children of the parent's neighbours (y-periodic, image m)
// that are not neighbours themselves; CSR (ptr, src, off, img), the same pairs
// grouped by offset in chunks of at most 16 (ptg, psr, pim, pof, cof, cbg,
// cen) and, for the tensor-core M2L, tiles of 128 target boxes.
struct M2LLists {
  std::vector<int> ptr, src, off, img, ptg, psr, pim, pof, cof, cbg, cen, tbox, tnoff, toffs, tsrc, timg;
  int ntile = 0;
};

static void build_m2l_lists(const Level& L, int l, int nr, bool tc, M2LLists& o) {
  const int nl = 1 << l, nlx = nr << l, np = nr << (l - 1);
  const int nne = (int)L.hne.size();
  // occupancy of the level's boxes on the (x, y) grid
  std::vector<unsigned char> occ((size_t)nlx * nl, 0);
  for (int b : L.hne) {
    int bx, by;
    box_xy(b, l, &bx, &by);
    occ[(size_t)by * nlx + bx] = 1;
  }
  std::vector<int>& ptr = o.ptr;
  std::vector<int>& src = o.src;
  std::vector<int>& off = o.off;
  std::vector<int>& img = o.img;
  ptr.assign(nne + 1, 0);
  src.reserve((size_t)27 * nne);
  off.reserve((size_t)27 * nne);
  img.reserve((size_t)27 * nne);
  for (int ti = 0; ti < nne; ++ti) {
    const int b = L.hne[ti];
    int ix, iy;
    box_xy(b, l, &ix, &iy);
    const int px = ix >> 1, py = iy >> 1;
    for (int pdx = -1; pdx <= 1; ++pdx) {
      const int qx = px + pdx;
      if (qx < 0 || qx >= np) continue;
      for (int pdy = -1; pdy <= 1; ++pdy) {
        const int qy = py + pdy;
        for (int cx = 0; cx < 2; ++cx)
          for (int cy = 0; cy < 2; ++cy) {
            const int sx = 2 * qx + cx, sy = 2 * qy + cy;
            const int dx = ix - sx, dy = iy - sy;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            const int syw = sy & (nl - 1);            // nl is a power of two
            if (!occ[(size_t)syw * nlx + sx]) continue;
            src.push_back(box_id(sx, syw, l));
            off.push_back((dx + 3) * 7 + (dy + 3));
            img.push_back((sy - syw) >> l);
          }
      }
    }
    ptr[ti + 1] = (int)src.size();
  }
  // the same pairs grouped by offset (a stable counting sort), cut into chunks
  // of at most 16 pairs (small chunks spread one level's translations over many blocks)
  const size_t n = src.size();
  int first[50] = {0};
  for (size_t e = 0; e < n; ++e) first[off[e] + 1]++;
  for (int q = 0; q < 49; ++q) first[q + 1] += first[q];
  o.ptg.resize(n);
  o.psr.resize(n);
  o.pim.resize(n);
  o.pof.resize(n);
  {
    int at[49];
    std::copy(first, first + 49, at);
    for (int ti = 0; ti < nne; ++ti)
      for (int e = ptr[ti]; e < ptr[ti + 1]; ++e) {
        const int q = at[off[e]]++;
        o.ptg[q] = L.hne[ti];
        o.psr[q] = src[e];
        o.pim[q] = img[e];
        o.pof[q] = off[e];
      }
  }
  for (int q = 0; q < 49; ++q)
    for (int b0 = first[q]; b0 < first[q + 1]; b0 += 16) {
      o.cof.push_back(q);
      o.cbg.push_back(b0);
      o.cen.push_back(std::min(b0 + 16, first[q + 1]));
    }
  if (tc) {
    // tensor-core tiles: 128 consecutive non-empty target boxes
    const int nt = (nne + 127) / 128;
    o.ntile = nt;
    o.tbox.assign((size_t)nt * 128, -1);
    o.tnoff.assign(nt, 0);
    o.toffs.assign((size_t)nt * 49, 0);
    o.tsrc.assign((size_t)nt * 49 * 128, -1);
    o.timg.assign((size_t)nt * 49 * 128, 0);
    for (int tile = 0; tile < nt; ++tile) {
      int slot[49];
      for (int q = 0; q < 49; ++q) slot[q] = -1;
      for (int r = 0; r < 128; ++r) {
        const size_t ti = (size_t)tile * 128 + r;
        if (ti >= L.hne.size()) break;
        o.tbox[ti] = L.hne[ti];
        for (int e = ptr[ti]; e < ptr[ti + 1]; ++e) {
          const int q = off[e];
          if (slot[q] < 0) {
            slot[q] = o.tnoff[tile]++;
            o.toffs[(size_t)tile * 49 + slot[q]] = q;
          }
          const size_t qq = ((size_t)tile * 49 + slot[q]) * 128 + r;
          o.tsrc[qq] = src[e];
          o.timg[qq] = img[e];
        }
      }
    }
  }
}

// Issues the launches of f on set-up stream i, ordered after everything issued
// so far on the main stream; the main stream waits for them at the join of
// build_plan (aux_ev).  While f runs, h->stream names stream i, so that the
// launchers, allocations and profiling events of f go there.
template <class F>
static pfmbem_status on_aux(pfmbem* h, int i, F&& f) {
  if (!h->aux[i]) CK(pool_stream(h->dev, &h->aux[i], i == 2));
  if (!h->aux_ev[i]) CK(pool_event(h->dev, &h->aux_ev[i]));
  if (!h->fork_ev) CK(pool_event(h->dev, &h->fork_ev));
  CK(cudaEventRecord(h->fork_ev, h->stream));
  CK(cudaStreamWaitEvent(h->aux[i], h->fork_ev, 0));
  cudaStream_t main_stream = h->stream;
  h->stream = h->aux[i];
  const pfmbem_status st = f();
  h->stream = main_stream;
  if (st != PFMBEM_OK) return st;
  CK(cudaEventRecord(h->aux_ev[i], h->aux[i]));
  return PFMBEM_OK;
}

// Regular polygon (equal chords, equal turning angles) of n elements from f0:
// rotating by one element maps the fiber onto itself.
static bool regular_polygon(const std::vector<double>& len, const std::vector<double2>& t, int f0, int n) {
  double hm = 0;
  for (int e = f0; e < f0 + n; ++e) hm += len[e];
  hm /= n;
  // the turn between consecutive unit tangents, as its (sine, cosine)
  double sn0 = 0, cs0 = 0;
  for (int q = 0; q < n; ++q) {
    const int e = f0 + q, e1 = q + 1 < n ? e + 1 : f0;
    if (std::fabs(len[e] - hm) > 1e-12 * hm) return false;
    const double sn = t[e].x * t[e1].y - t[e].y * t[e1].x, cs = t[e].x * t[e1].x + t[e].y * t[e1].y;
    if (q == 0) {
      sn0 = sn;
      cs0 = cs;
    } else if (std::fabs(sn - sn0) > 1e-12 || std::fabs(cs - cs0) > 1e-12) {
      return false;
    }
  }
  return true;
}

#include "tri_plan.h"

static pfmbem_status build_plan(pfmbem* h, const int* npf, const double* nodes) {
  const double t0 = now_ms();
  const int M = h->M;
  const double H = h->H, k = h->k;
  // ---------------------------------------------------- elements (original order)
  std::vector<int> foff(M + 1, 0);
  for (int i = 0; i < M; ++i) {
    if (npf[i] < 3) return fail(h, PFMBEM_EGEOM, "fiber " + std::to_string(i) + " has fewer than 3 nodes");
    foff[i + 1] = foff[i] + npf[i];
  }
  const int E = foff[M];
  h->E = E;
  h->hfib_off = foff;
  std::vector<double2> c(E), t(E), nu(E);
  std::vector<double> len(E);
  std::vector<int> fib(E);
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, hmax = 0, hmin = 1e300;
  for (int i = 0; i < M; ++i) {
    double area = 0;
    const int n = npf[i];
    h->max_fiber = std::max(h->max_fiber, n);
    for (int j = 0; j < n; ++j) {
      const double* a = nodes + 2 * (foff[i] + j);
      const double* b = nodes + 2 * (foff[i] + (j + 1) % n);
      if (!std::isfinite(a[0]) || !std::isfinite(a[1])) return fail(h, PFMBEM_EGEOM, "non-finite node");
      const int e = foff[i] + j;
      double dx = b[0] - a[0], dy = b[1] - a[1];
      double L = std::sqrt(dx * dx + dy * dy);      // node coordinates are O(H): no overflow concern
      if (!(L > 0)) return fail(h, PFMBEM_EGEOM, "zero-length element " + std::to_string(e));
      c[e] = double2{0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1])};
      t[e] = double2{dx / L, dy / L};
      nu[e] = double2{dy / L, -dx / L};
      len[e] = L;
      fib[e] = i;
      area += a[0] * b[1] - a[1] * b[0];
      xmin = std::min(xmin, a[0]); xmax = std::max(xmax, a[0]);
      ymin = std::min(ymin, a[1]); ymax = std::max(ymax, a[1]);
      hmax = std::max(hmax, L);
      hmin = std::min(hmin, L);
    }
    if (!(area > 0)) return fail(h, PFMBEM_EGEOM, "fiber " + std::to_string(i) + " is not counter-clockwise");
  }
  // a block wider than H along x takes a row of root squares of side H (Sec. 2
  // allows any width L; the y-period H sets the root's side)
  {
    const int nr = std::max(1, (int)std::ceil((xmax - xmin) / H - 1e-12));
    if (nr > kMaxRoots && h->opt.tree != 1) return fail(h, PFMBEM_EGEOM, "block wider than 4 H along x");
    h->nroot = nr;
  }
  // fiber centre (mean of the nodes) and mean radius, for the learned warm start
  h->hfib_geo.assign(3 * (size_t)M, 0.0);
  for (int i = 0; i < M; ++i) {
    double sx = 0, sy = 0, sr = 0;
    const int n = npf[i];
    for (int j = 0; j < n; ++j) {
      sx += nodes[2 * (foff[i] + j)];
      sy += nodes[2 * (foff[i] + j) + 1];
    }
    sx /= n;
    sy /= n;
    for (int j = 0; j < n; ++j) {
      const double dx = nodes[2 * (foff[i] + j)] - sx, dy = nodes[2 * (foff[i] + j) + 1] - sy;
      sr += std::sqrt(dx * dx + dy * dy);
    }
    h->hfib_geo[3 * i] = sx;
    h->hfib_geo[3 * i + 1] = sy;
    h->hfib_geo[3 * i + 2] = sr / n;
  }
  if (h->opt.tree == 1) return build_plan_tri(h, nodes, foff, c, t, nu, len, fib, hmax, t0);
  if (h->opt.tree != 0) return fail(h, PFMBEM_EINVAL, "tree must be 0 (square) or 1 (triangle)");
  if (0.5 * k * hmax > 4.0) return fail(h, PFMBEM_EINVAL, "elements longer than 8/k");
  // ---------------------------------------------------- root box and wrapping
  h->x0 = 0.5 * (xmin + xmax) - 0.5 * h->nroot * H;
  h->y0 = 0.5 * (ymin + ymax) - 0.5 * H;
  const int NR = h->nroot;
  std::vector<int> m0(E);
  std::vector<double2> cw(E);
  for (int e = 0; e < E; ++e) {
    int m = (int)std::floor((c[e].y - h->y0) / H);
    m0[e] = m;
    cw[e] = double2{c[e].x, c[e].y - m * H};
  }
  // optional set-up timing on stderr: PFMBEM_TIMING=1 wall time per section
  // (the stream is synchronised at every mark), =2 host time only (no sync),
  // =3 trace: timing events on the set-up streams, reported at the end
  const char* tenv = std::getenv("PFMBEM_TIMING");
  h->trace_on = tenv != nullptr && std::strcmp(tenv, "3") == 0;
  const bool timing = tenv != nullptr && !h->trace_on;
  const bool tsync = timing && std::strcmp(tenv, "2") != 0;
  double tmark = now_ms();
  auto mark = [&](const char* what) {
    trace(h, h->astream ? h->astream : h->stream, what);
    if (!timing) return;
    if (tsync) cudaStreamSynchronize(h->astream ? h->astream : h->stream);
    const double t = now_ms();
    std::fprintf(stderr, "pfmbem setup %-22s %8.2f ms\n", what, t - tmark);
    tmark = t;
  };
  mark("elements");
  h->ub_on = true;                 // tables below go up in a few batched copies
  pin_acquire(h);
  // ---------------------------------------------------- depth
  const int leaf_max = h->opt.leaf_max > 0 ? h->opt.leaf_max : 64;
  int D = h->opt.depth;
  // box coordinates of every midpoint at the finest admissible depth (10); the
  // box at depth D is the same pair shifted right by 10 - D bits
  // and its Morton code: the code of the depth-D box is a prefix of it
  std::vector<int> m10(E);
  {
    // (a value below 0 truncates to 0 like its floor clamps to 0)
    const double r10 = 1024.0 / H;
    for (int e = 0; e < E; ++e) {
      const int ix = std::min(std::max((int)((cw[e].x - h->x0) * r10), 0), 1024 * NR - 1);
      const int iy = std::min(std::max((int)((cw[e].y - h->y0) * r10), 0), 1023);
      m10[e] = box_id(ix, iy, 10);
    }
  }
  // box occupancy at depth 8 in one pass, then at every coarser depth by
  // summing the four Morton-consecutive children: cnt[l][b], l <= 8
  constexpr int DH = 8;
  std::vector<std::vector<int>> cnt(DH + 1);
  cnt[DH].assign((size_t)NR << (2 * DH), 0);
  for (int e = 0; e < E; ++e) cnt[DH][m10[e] >> (2 * (10 - DH))]++;
  for (int l = DH - 1; l >= 0; --l) {
    cnt[l].resize((size_t)NR << (2 * l));
    const int* c1 = cnt[l + 1].data();
    for (size_t b = 0; b < cnt[l].size(); ++b) cnt[l][b] = c1[4 * b] + c1[4 * b + 1] + c1[4 * b + 2] + c1[4 * b + 3];
  }
  if (D <= 0) {
    for (D = 2; D < 10; ++D) {
      int mx = 0;
      if (D <= DH) {
        for (int v : cnt[D]) mx = std::max(mx, v);
      } else {
        std::vector<int> c((size_t)NR << (2 * D), 0);
        for (int e = 0; e < E; ++e) mx = std::max(mx, ++c[m10[e] >> (2 * (10 - D))]);
      }
      if (mx <= leaf_max) break;
    }
  }
  if (D < 2 || D > 10) return fail(h, PFMBEM_EINVAL, "depth must be in [2, 10]");
  h->D = D;
  // ---------------------------------------------------- sort by leaf Morton key (stable counting sort)
  std::vector<int> key(E), perm(E), pos(E);
  for (int e = 0; e < E; ++e) key[e] = m10[e] >> (2 * (10 - D));
  if (D > DH) {
    cnt.resize(D + 1);
    for (int l = DH + 1; l <= D; ++l) {
      cnt[l].assign((size_t)NR << (2 * l), 0);
      for (int e = 0; e < E; ++e) cnt[l][m10[e] >> (2 * (10 - l))]++;
    }
  }
  {
    std::vector<int> start(((size_t)NR << (2 * D)) + 1, 0);
    for (size_t b = 0; b + 1 < start.size(); ++b) start[b + 1] = start[b] + cnt[D][b];
    for (int e = 0; e < E; ++e) perm[start[key[e]]++] = e;
  }
  for (int s = 0; s < E; ++s) pos[perm[s]] = s;
  // ---------------------------------------------------- levels
  for (int l = 0; l <= D; ++l) {
    Level& L = h->lev[l];
    L.nbox = NR << (2 * l);
    L.d = H / (1 << l);
    L.hbegin.resize(L.nbox);
    L.hend.resize(L.nbox);
    const int* cl = cnt[l].data();
    int acc = 0;
    for (int b = 0; b < L.nbox; ++b) {
      L.hbegin[b] = acc;
      acc += cl[b];
      L.hend[b] = acc;
      if (cl[b] > 0) L.hne.push_back(b);
    }
    L.nne = (int)L.hne.size();
    // expansion order
    double x = k * L.d * std::sqrt(2.0);
    // p_min = 24: the fine levels' translations (kd << 1) converge geometrically,
    // by about 0.4 per order for the nearest well-separated boxes (Table 1, L = 0),
    // so p_min sets the FMM's error on smooth densities: measured against the
    // oracle on the 8x8 hexagon block's solution, 1.6e-6 at 15, 3.8e-8 at 20,
    // 6.9e-10 at 24
    int pmin = h->opt.p_min > 0 ? h->opt.p_min : 24;
    int p = h->opt.p > 0 ? h->opt.p : (int)std::ceil(x + 1.8 * std::pow(10.0, 2.0 / 3.0) * std::cbrt(x));
    p = std::max(p, h->opt.p > 0 ? 1 : pmin);
    if (p > PF_PMAX) return fail(h, PFMBEM_EINVAL, "expansion order above the library limit (128); use more levels");
    L.p = p;
    L.P = 2 * p + 1;
    // the FP32 product's order: the same rule with the lower bound p_min_mixed
    // (0 = 18: its truncation, ~0.4^p as for p_min, stays near the FP32 rounding)
    {
      const int pm32 = h->opt.p_min_mixed > 0 ? h->opt.p_min_mixed : 18;
      const int rule = (int)std::ceil(x + 1.8 * std::pow(10.0, 2.0 / 3.0) * std::cbrt(x));
      L.p32 = h->opt.p > 0 ? p : std::min(p, std::max(rule, pm32));
    }
    L.sigma = k * L.d / std::sqrt(2.0);
    L.w.assign(L.P, 1.0);
    double wn = 1.0;
    for (int n = 1; n <= p; ++n) {
      wn *= L.sigma / n;
      L.w[p + n] = wn;
      L.w[p - n] = wn;
    }
    h->info.p[l] = p;
  }
  if (NR > 1) {
    // the super root over the row: its centre C, radius R_s (the half-diagonal of
    // the nr H x H row), the first image row m0 it takes (m0 H >= 3 R_s: the super
    // M2L's ratio 2 R_s / (m0 H) stays at or below 2/3) and its order (the levels'
    // rule for a box of diagonal 2 R_s)
    if (h->opt.launch != 0 || h->opt.near_mode != 0 || h->opt.m2l_mode == 2)
      return fail(h, PFMBEM_EINVAL, "blocks wider than H need the cached single-launch product (default options)");
    h->wide_cx = h->x0 + 0.5 * NR * H;
    h->wide_cy = h->y0 + 0.5 * H;
    h->wide_rs = 0.5 * H * std::sqrt((double)NR * NR + 1.0);
    h->wide_m0 = (int)std::ceil(3.0 * h->wide_rs / H - 1e-12);
    const double x = 2.0 * k * h->wide_rs;
    // at least the order at which the super M2L's ratio 2 R_s / (m0 H), to that
    // power, falls to 1e-11
    const int pratio = (int)std::ceil(std::log(1e-11) / std::log(2.0 * h->wide_rs / (h->wide_m0 * H)));
    const int ps = std::max({(int)std::ceil(x + 1.8 * std::pow(10.0, 2.0 / 3.0) * std::cbrt(x)), h->lev[0].p, pratio});
    if (ps > PF_PMAX) return fail(h, PFMBEM_EINVAL, "block too wide for this frequency (super-root order above 128)");
    h->wide_ps = ps;
  }
  mark("depth, sort, levels");
  // the M2L lists depend on the tree alone: a worker thread builds them while
  // the set-up below goes on (they are uploaded where the second stream starts)
  // M2L on the tensor cores in the single-launch FP32 product: by default at
  // the levels with at least tc_min_boxes non-empty boxes (below that the
  // tiles of 128 targets run mostly empty); m2l_mode 2: every level, 1: none.
  // Only where the product's order there gives 2P <= 80 (the operands' shared
  // memory).  PFMBEM_TC_MIN_BOXES overrides the threshold, for measurement.
  {
    static const char* tmb = std::getenv("PFMBEM_TC_MIN_BOXES");
    const int tc_min_boxes = tmb ? std::max(1, std::atoi(tmb)) : 1024;
    const bool fusable = h->opt.near_mode == 0 && h->max_fiber <= 1024 && h->opt.launch == 0;
    for (int l = 1; l <= D; ++l) {
      Level& L = h->lev[l];
      const int pu = D >= 3 && NR == 1 ? std::min(L.p, std::max(1, L.p32)) : L.p;
      L.tc_fused = fusable && h->opt.m2l_mode != 1 && tc_kpad(2 * pu + 1) <= 80 &&
                   (h->opt.m2l_mode == 2 ? L.nne > 0 : L.nne >= tc_min_boxes);
    }
  }
  std::vector<M2LLists> m2l(D + 1);
  std::future<void> m2l_lists = std::async(std::launch::async, [h, D, &m2l]() {
    for (int l = 1; l <= D; ++l)
      build_m2l_lists(h->lev[l], l, h->nroot, h->opt.m2l_mode == 2 || h->lev[l].tc_fused, m2l[l]);
  });
  // ---------------------------------------------------- lists
  const int nD = 1 << D, nDx = NR << D;
  std::vector<int64_t> nc_base;
  std::vector<int> nc_sbase(1, 0);
  std::vector<int> nl_ptr(1, 0), nl_src, nl_img;      // near lists of the leaves: source leaf, image m
  {
    Level& Lf = h->lev[D];
    std::vector<int>& ptr = nl_ptr;
    std::vector<int>& src = nl_src;
    std::vector<int>& img = nl_img;
    for (int b : Lf.hne) {
      int ix, iy;
      box_xy(b, D, &ix, &iy);
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
          int sx = ix + dx, sy = iy + dy;
          if (sx < 0 || sx >= nDx) continue;
          int syw = ((sy % nD) + nD) % nD;
          int m = (sy - syw) / nD;
          int sb = box_id(sx, syw, D);
          if (Lf.hend[sb] > Lf.hbegin[sb]) { src.push_back(sb); img.push_back(m); }
        }
      ptr.push_back((int)src.size());
    }
    CK(cudaSuccess);
    pfmbem_status st;
    if ((st = upload(h, &h->nl_ptr, ptr)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->nl_src, src)) != PFMBEM_OK) return st;
    if ((st = upload(h, &h->nl_img, img)) != PFMBEM_OK) return st;
    // near-field pair statistics (the cache build counts them on the GPU)
    int64_t pairs = 0, quad = 0;
    for (size_t li = 0; h->opt.near_mode != 0 && li < Lf.hne.size(); ++li) {
      int b = Lf.hne[li];
      for (int s = Lf.hbegin[b]; s < Lf.hend[b]; ++s)
        for (int e = ptr[li]; e < ptr[li + 1]; ++e) {
          int sb = src[e];
          for (int f = Lf.hbegin[sb]; f < Lf.hend[sb]; ++f) {
            if (f == s && img[e] == 0) continue;
            int eo = perm[f], so = perm[s];
            double dx = cw[so].x - cw[eo].x, dy = cw[so].y - (cw[eo].y + img[e] * H);
            double q = std::hypot(dx, dy) / len[eo];
            pairs++;
            quad += gl_order_host(q, g_thr64);
          }
        }
    }
    h->info.near_pairs = pairs;
    h->info.near_quad = quad;
    // layout of the cached near field: per leaf, its concatenated source list
    // (filled on the device from the leaf's near list) and a dense
    // [targets][sources] array of 2x2 complex blocks
    int64_t acc = 0;
    nc_sbase.reserve(Lf.hne.size() + 1);
    nc_base.reserve(Lf.hne.size());
    for (size_t li = 0; li < Lf.hne.size(); ++li) {
      int b = Lf.hne[li];
      int ns = 0;
      for (int e = ptr[li]; e < ptr[li + 1]; ++e) ns += Lf.hend[src[e]] - Lf.hbegin[src[e]];
      nc_sbase.push_back(nc_sbase.back() + ns);
      h->nc_maxns = std::max(h->nc_maxns, ns);
      h->leaf_maxn = std::max(h->leaf_maxn, Lf.hend[b] - Lf.hbegin[b]);
      nc_base.push_back(acc);
      acc += 4 * (int64_t)(Lf.hend[b] - Lf.hbegin[b]) * ns;
    }
    h->nc_blocks = acc / 4;
  }
  // fiber-local statistics (the cache build counts them on the GPU)
  {
    int64_t pairs = 0, quad = 0;
    for (int i = 0; h->opt.near_mode != 0 && i < M; ++i)
      for (int e = foff[i]; e < foff[i + 1]; ++e)
        for (int f = foff[i]; f < foff[i + 1]; ++f) {
          if (f == e) continue;
          double q = std::hypot(c[e].x - c[f].x, c[e].y - c[f].y) / len[f];
          pairs++;
          quad += gl_order_host(q, g_thr64);
        }
    h->info.fiber_pairs = pairs;
    h->info.fiber_quad = quad;
  }
  // P2M Gauss nodes: elements outside the near field are at least one leaf
  // side minus half an element length away.
  {
    double qfar = std::max(1.0, h->lev[D].d / hmax - 1.0);
    h->g_far = gl_order_host(qfar, g_thr64);
    h->g_far_f = gl_order_host(qfar, g_thr32);
  }
  // box ranges and expansion weights of every level
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
  }
  mark("near lists");
  // ---------------------------------------------------- element arrays
  {
    // the tree-ordered copies (wrapped midpoints, alpha^{-m0}, leaf keys) are
    // gathered on the device from the original-order arrays
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
  if (!h->s_c || !h->s_t || !h->s_nu || !h->s_h || !h->s_ph || !h->s_m0 || !h->s_leaf)
    return fail(h, PFMBEM_ENOMEM, "device allocation failed (element arrays)");
  h->self4 = dalloc<cplx>(h, (size_t)4 * E);
  h->dens = dalloc<cplx>(h, (size_t)2 * E);
  h->U = dalloc<cplx>(h, (size_t)2 * E);
  h->stage_in = dalloc<cplx>(h, (size_t)2 * E);
  h->stage_out = dalloc<cplx>(h, (size_t)2 * E);
  h->dev_rhs = dalloc<cplx>(h, (size_t)2 * E);
  if (!h->self4 || !h->dens || !h->U || !h->stage_in || !h->stage_out || !h->dev_rhs)
    return fail(h, PFMBEM_ENOMEM, "device allocation failed (work buffers)");
  {
    pfmbem_status st;
    if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
  }
  CK(k_sort_elements(h));
  h->tab_err = dalloc<int>(h, 1);
  if (!h->tab_err) return fail(h, PFMBEM_ENOMEM, "device allocation failed");
  CK(cudaMemsetAsync(h->tab_err, 0, sizeof(int), h->stream));
  CK(k_self_terms(h));
  mark("element arrays, self terms");
  // ---------------------------------------------------- lattice sums + root operator
  if (!h->side_ev) CK(pool_event(h->dev, &h->side_ev));
  {
    // on their own stream: nothing else of the set-up waits for them until the join
    pfmbem_status st = on_aux(h, 0, [&]() -> pfmbem_status {
      Level& R = h->lev[0];
      const int p0 = R.p, P0 = R.P, jmax = 2 * p0;
      if (h->nroot > 1) {
        // a row of root squares: the operator between all roots (k_wide_top)
        const int nr = h->nroot, ps = h->wide_ps, Ps = 2 * ps + 1;
        h->root = dalloc<cplx>(h, (size_t)nr * P0 * nr * P0);
        h->rootf = dalloc<cplxf>(h, (size_t)P0 * P0);
        double2* dv = dalloc<double2>(h, 2 * nr);
        h->wide_w = dalloc<double>(h, Ps);
        h->wide_A = dalloc<cplx>(h, (size_t)nr * P0 * Ps);
        h->wide_B = dalloc<cplx>(h, (size_t)nr * Ps * P0);
        h->wide_Rs = dalloc<cplx>(h, (size_t)Ps * Ps);
        h->wide_ML = dalloc<cplx>(h, 2 * (size_t)Ps);
        cplx* S = dalloc<cplx>(h, (size_t)2 * ps + 1);
        cplx* X = dalloc<cplx>(h, (size_t)nr * Ps * P0);
        if (!h->root || !h->rootf || !dv || !h->wide_w || !h->wide_A || !h->wide_B || !h->wide_Rs || !h->wide_ML ||
            !S || !X)
          return fail(h, PFMBEM_ENOMEM, "device allocation failed (root row)");
        std::vector<double2> hv(2 * nr);
        for (int i = 0; i < nr; ++i) {
          const double cx = h->x0 + (i + 0.5) * H, cy = h->y0 + 0.5 * H;
          hv[i] = double2{cx, cy};
          hv[nr + i] = double2{cx - h->wide_cx, cy - h->wide_cy};
        }
        // the super root's weights w_n = sigma^|n| / |n|!, sigma = k R_s, as the levels'
        std::vector<double> w(Ps, 1.0);
        double wn = 1.0;
        for (int n = 1; n <= ps; ++n) {
          wn *= k * h->wide_rs / n;
          w[ps + n] = w[ps - n] = wn;
        }
        // (pageable sources: the copies have left the vectors when the calls return)
        CK(cudaMemcpyAsync(dv, hv.data(), sizeof(double2) * 2 * nr, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->wide_w, w.data(), sizeof(double) * Ps, cudaMemcpyHostToDevice, h->stream));
        CK(k_wide_top(h, dv, S, X));
        trace(h, h->stream, "aux0: root row operators done");
        return PFMBEM_OK;
      }
      cplx* Sd = dalloc<cplx>(h, jmax + 1);
      h->root = dalloc<cplx>(h, (size_t)P0 * P0);
      h->rootf = dalloc<cplxf>(h, (size_t)P0 * P0);
      if (!Sd || !h->root || !h->rootf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (lattice sums)");
      CK(k_lattice_sums(h, jmax, h->lattice_q, Sd));
      // root translation R[a][n] = w_a S_{|n-a|} w_n, built on the device
      CK(k_root_operator(h, p0, R.w_dev, Sd));
      trace(h, h->stream, "aux0: lattice sums, root done");
      return PFMBEM_OK;
    });
    if (st != PFMBEM_OK) return st;
  }
  mark("lattice sums, root");
  // the second stream starts after everything uploaded so far (level weights)
  if (!h->pre_ev) CK(pool_event(h->dev, &h->pre_ev));
  CK(cudaEventRecord(h->pre_ev, h->stream));
  // ---------------------------------------------------- translation tables
  // One FP64 and one FP32 arena hold every level's expansions and operators
  // (sub-arrays aligned to 256 bytes); the operators are built on the device,
  // on the second stream as soon as the level weights are up.
  if (!h->side) CK(pool_stream(h->dev, &h->side));
  CK(cudaStreamWaitEvent(h->side, h->pre_ev, 0));
  h->astream = h->side;
  {
    auto up16 = [](size_t n) { return (n + 15) & ~(size_t)15; };
    size_t n64 = 0, n32 = 0;
    for (int l = 0; l <= D; ++l) {
      const Level& L = h->lev[l];
      const size_t ex = up16((size_t)L.nbox * L.P);
      const size_t tm = l >= 1 ? up16((size_t)49 * L.P * L.P) : 0;
      const size_t mm = l < D ? up16((size_t)4 * L.P * h->lev[l + 1].P) : 0;
      n64 += 2 * ex + 2 * tm + 2 * mm;
      n32 += 2 * up16(ex) + 3 * up16(tm) + 4 * up16(mm);
    }
    cplx* a64 = dalloc<cplx>(h, n64);
    cplxf* a32 = dalloc<cplxf>(h, n32);
    if (!a64 || !a32) return fail(h, PFMBEM_ENOMEM, "device allocation failed (expansions, tables)");
    TableLevels tl{};
    for (int l = 0; l <= D; ++l) {
      Level& L = h->lev[l];
      const int P = L.P;
      const size_t ex = up16((size_t)L.nbox * P);
      L.M = a64; a64 += ex;
      L.L = a64; a64 += ex;
      L.Mf = a32; a32 += ex;
      L.Lf = a32; a32 += ex;
      tl.p[l] = L.p;
      tl.d[l] = L.d;
      tl.w[l] = L.w_dev;
      if (l >= 1) {
        const size_t tm = up16((size_t)49 * P * P);
        L.m2l = a64; a64 += tm;
        L.m2lt = a64; a64 += tm;
        L.m2lf = a32; a32 += tm;
        L.m2ltf = a32; a32 += tm;
        L.m2ltl = a32; a32 += tm;
        tl.T[l] = L.m2l; tl.Tt[l] = L.m2lt; tl.Tf[l] = L.m2lf; tl.Ttf[l] = L.m2ltf; tl.Ttl[l] = L.m2ltl;
        // tensor-core operators: the per-stage kernels' (full order), the
        // single-launch FP32 product's (its order, interleaved layout)
        if (tc_kpad(P) <= 128 && h->opt.m2l_mode == 2 && h->opt.launch == 1) {
          const int kp = tc_kpad(P);
          L.tc_B = dalloc<uint16_t>(h, (size_t)49 * 3 * kp * kp);
          if (!L.tc_B) return fail(h, PFMBEM_ENOMEM, "device allocation failed (tensor-core operators)");
        }
        if (L.tc_fused) {
          const int pu = D >= 3 && NR == 1 ? std::min(L.p, std::max(1, L.p32)) : L.p;
          const int kp = tc_kpad(2 * pu + 1);
          L.tc_Bf = dalloc<uint16_t>(h, (size_t)49 * 3 * kp * kp);
          if (!L.tc_Bf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (tensor-core operators)");
        }
      }
      if (l < D) {
        const size_t mm = up16((size_t)4 * P * h->lev[l + 1].P);
        L.m2m = a64; a64 += mm;
        L.l2l = a64; a64 += mm;
        L.m2mf = a32; a32 += mm;
        L.m2ml = a32; a32 += mm;
        L.l2lf = a32; a32 += mm;
        L.l2ll = a32; a32 += mm;
        tl.A[l] = L.m2m; tl.B[l] = L.l2l; tl.Af[l] = L.m2mf; tl.Bf[l] = L.l2lf; tl.Al[l] = L.m2ml;
        tl.Bl[l] = L.l2ll;
      }
    }
    CK(k_tables(h, tl, h->astream ? h->astream : h->stream));
    trace(h, h->astream ? h->astream : h->stream, "side: translation tables done");
  }
  h->astream = nullptr;

  // ---------------------------------------------------- near-field / fiber caches
  // The element integrals of the caches run on the GPU while the host builds
  // the M2L lists and translation tables on a second stream; the streams join
  // before the P2M/L2P caches.
  bool cache = false;
  if (h->opt.near_mode == 0 && h->max_fiber <= 1024) {
    std::vector<int64_t> fbase(M, 0);
    std::vector<int> chunks, circ(M, 0);
    int64_t acc = 0;
    for (int i = 0; i < M; ++i) {
      // regular polygon: its block is circulant and is stored as the row pair of
      // its first element
      circ[i] = regular_polygon(len, t, foff[i], foff[i + 1] - foff[i]) ? 1 : 0;
      fbase[i] = acc;
      const int n2 = 2 * (foff[i + 1] - foff[i]);
      acc += circ[i] ? (int64_t)2 * n2 : (int64_t)n2 * n2;
      for (int r = 0; r < n2; r += 32) {
        chunks.push_back(i);
        chunks.push_back(r);
        chunks.push_back(std::min(r + 32, n2));
      }
    }
    h->fb_entries = acc;
    h->hcirc = circ;
    const double bytes = (double)(4 * h->nc_blocks + acc) * (sizeof(cplx) + sizeof(cplxf));
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    if (bytes < 0.5 * (double)freeb) {
      pfmbem_status st;
      // P2M/L2P caches (element geometry only) on their own stream
      st = on_aux(h, 1, [&]() -> pfmbem_status {
        const size_t nc = (size_t)E * 2 * h->lev[D].P;
        h->p2m_c = dalloc<cplx>(h, nc);
        h->l2p_c = dalloc<cplx>(h, nc);
        h->p2m_cf = dalloc<cplxf>(h, nc);
        h->p2m_cl = dalloc<cplxf>(h, nc);
        h->l2p_cl = dalloc<cplxf>(h, nc);
        if (!h->p2m_cl || !h->l2p_cl) return fail(h, PFMBEM_ENOMEM, "device allocation failed (P2M/L2P caches)");
        h->l2p_cf = dalloc<cplxf>(h, nc);
        h->densf = dalloc<cplxf>(h, (size_t)2 * E);
        h->Uf = dalloc<cplxf>(h, (size_t)2 * E);
        if (!h->p2m_c || !h->l2p_c || !h->p2m_cf || !h->l2p_cf || !h->densf || !h->Uf)
          return fail(h, PFMBEM_ENOMEM, "device allocation failed (P2M/L2P caches)");
        trace(h, h->stream, "aux1: P2M/L2P caches start");
        CK(k_build_fmm_caches(h));
        trace(h, h->stream, "aux1: P2M/L2P caches done");
        return PFMBEM_OK;
      });
      if (st != PFMBEM_OK) return st;
      if ((st = upload(h, &h->nc_base, nc_base)) != PFMBEM_OK) return st;
      if ((st = upload(h, &h->nc_sbase, nc_sbase)) != PFMBEM_OK) return st;
      h->nc_src = dalloc<int>(h, (size_t)std::max(nc_sbase.back(), 1));
      h->nc_img = dalloc<int>(h, (size_t)std::max(nc_sbase.back(), 1));
      if (!h->nc_src || !h->nc_img) return fail(h, PFMBEM_ENOMEM, "device allocation failed (near sources)");
      if ((st = upload(h, &h->fb_base, fbase)) != PFMBEM_OK) return st;
      if ((st = upload(h, &h->fb_circ, circ)) != PFMBEM_OK) return st;
      if ((st = upload(h, &h->fb_chunk, chunks)) != PFMBEM_OK) return st;
      std::vector<int> rows;
      for (int i = 0; i < M; ++i)
        for (int e = foff[i]; e < (circ[i] ? foff[i] + 1 : foff[i + 1]); ++e) rows.push_back(e);
      h->nfb_rows = (int)rows.size();
      if ((st = upload(h, &h->fb_rows, rows)) != PFMBEM_OK) return st;
      // k tables of the regular-polygon fibers and the wrap shift of every element
      std::vector<int64_t> kbase(M, -1);
      int64_t kacc = 0;
      for (int i = 0; i < M; ++i)
        if (circ[i]) {
          kbase[i] = kacc;
          kacc += foff[i + 1] - foff[i];
        }
      if ((st = upload(h, &h->kt_base, kbase)) != PFMBEM_OK) return st;
      if ((st = build_pair_tables(h, nodes, foff, fib, m0, perm, nl_ptr, nl_src, nl_img)) != PFMBEM_OK) return st;
      h->kt_val = dalloc<cplx>(h, (size_t)4 * kacc);
      h->kt_sval = dalloc<cplx>(h, (size_t)4 * kacc);
      h->kt_svalf = dalloc<cplxf>(h, (size_t)4 * kacc);
      h->kt_svall = dalloc<cplxf>(h, (size_t)4 * kacc);
      if (!h->kt_sval || !h->kt_svalf || !h->kt_svall)
        return fail(h, PFMBEM_ENOMEM, "device allocation failed (fiber k tables)");
      if (!h->kt_val) return fail(h, PFMBEM_ENOMEM, "device allocation failed (fiber k tables)");
      h->nchunk = (int)chunks.size() / 3;
      // queue of the near pairs integrated directly: every block in the worst case
      h->nq_cap = (unsigned)std::min<int64_t>(h->nc_blocks, (int64_t)0xFFFFFFFFu);
      h->nq = dalloc<unsigned long long>(h, std::max<size_t>(h->nq_cap, 1));
      h->nq_len = dalloc<unsigned>(h, 1);
      if (!h->nq || !h->nq_len) return fail(h, PFMBEM_ENOMEM, "device allocation failed (near queue)");
      // (FP64 near blocks: formed from the double-float pair on first use, k_near64)
      h->nc_valf = dalloc<cplxf>(h, (size_t)(4 * h->nc_blocks));
      h->nc_vall = dalloc<cplxf>(h, (size_t)(4 * h->nc_blocks));
      h->dens_dd = dalloc<cplxf>(h, (size_t)4 * E);
      if (!h->nc_vall || !h->dens_dd) return fail(h, PFMBEM_ENOMEM, "device allocation failed (near-field caches)");
      h->fb_val = dalloc<cplx>(h, (size_t)acc);
      h->fb_valf = dalloc<cplxf>(h, (size_t)acc);
      h->stat_dev = dalloc<unsigned long long>(h, 4);
      h->tc_err = dalloc<int>(h, 1);
      if (!h->tc_err) return fail(h, PFMBEM_ENOMEM, "device allocation failed");
      CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
      if (!h->nc_valf || !h->fb_val || !h->fb_valf || !h->stat_dev)
        return fail(h, PFMBEM_ENOMEM, "device allocation failed (near-field caches)");
      CK(cudaMemsetAsync(h->stat_dev, 0, 4 * sizeof(unsigned long long), h->stream));
      if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
      mark("cache allocation");
      // the near-field chain (the longest of the set-up) on its own stream of
      // the highest priority; the same-fiber blocks here beside it
      if (!h->ktab_ev) CK(pool_event(h->dev, &h->ktab_ev));
      st = on_aux(h, 2, [&]() -> pfmbem_status {
        CK(k_build_caches(h, h->ktab_ev));
        return PFMBEM_OK;
      });
      if (st != PFMBEM_OK) return st;
      CK(k_build_fiber_blocks(h));
      cache = true;
      // the fiber symbols and the preconditioner go to the GPU now, ahead of
      // the host's M2L lists
      h->cached = true;
      if (h->opt.launch == 0) {
        // fibers applied by FFT (regular polygons with 2^j elements, 8 <= N <= 1024)
        // and the row chunks of the others
        std::vector<int> fft, zchunk;
        std::vector<int64_t> fhb(M, -1);
        const std::vector<int>& circh = h->hcirc;
        int64_t fa = 0;
        for (int i = 0; i < M; ++i) {
          const int n = foff[i + 1] - foff[i];
          if (circh[i] && n >= 8 && n <= 1024 && (n & (n - 1)) == 0) {
            fft.push_back(i);
            fhb[i] = fa;
            fa += n;
          } else {
            for (int r = 0; r < 2 * n; r += 32) {
              zchunk.push_back(i);
              zchunk.push_back(r);
              zchunk.push_back(std::min(r + 32, 2 * n));
            }
          }
        }
        h->fz_nfft = (int)fft.size();
        h->fz_nchunk = (int)zchunk.size() / 3;
        if ((st = upload(h, &h->fz_fft, fft)) != PFMBEM_OK) return st;
        if ((st = upload(h, &h->fz_chunk, zchunk)) != PFMBEM_OK) return st;
        {
          // (fiber, row) of every row applied by rows, for the FP32 product's row sums
          std::vector<int> rf;
          for (size_t c = 0; c + 2 < zchunk.size(); c += 3)
            for (int r = zchunk[c + 1]; r < zchunk[c + 2]; ++r) {
              rf.push_back(zchunk[c]);
              rf.push_back(r);
            }
          h->fz_nrowsum = (int)(rf.size() / 2);
          if (h->fz_nrowsum > 0 && (st = upload(h, &h->fz_rowfib, rf)) != PFMBEM_OK) return st;
        }
        if ((st = upload(h, &h->fh_base, fhb)) != PFMBEM_OK) return st;
        std::vector<cplx> twh(512);
        for (int j = 0; j < 512; ++j) twh[j] = cplx{std::cos(2.0 * M_PI * j / 1024.0), std::sin(2.0 * M_PI * j / 1024.0)};
        if ((st = upload(h, &h->tw, twh)) != PFMBEM_OK) return st;
        if ((st = upload(h, &h->twf, to_float(twh))) != PFMBEM_OK) return st;
        if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
        h->fh_val = dalloc<cplx>(h, (size_t)4 * fa);
        h->fh_valf = dalloc<cplxf>(h, (size_t)4 * fa);
        if (!h->fh_val || !h->fh_valf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (fiber symbols)");
        CK(k_fiber_symbols(h));
        CK(cudaStreamWaitEvent(h->stream, h->ktab_ev, 0));   // the preconditioner reads the k tables
        if (h->opt.precond == 0 && h->fz_nfft > 0) {
          h->pc_val = dalloc<cplx>(h, (size_t)4 * fa);
          h->pc_valf = dalloc<cplxf>(h, (size_t)4 * fa);
          if (!h->pc_val || !h->pc_valf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (preconditioner)");
          CK(k_precond_symbols(h));
        }
        if (h->opt.precond == 0) {
          // the other regular polygons: preconditioner kept as a circulant row pair
          std::vector<int> prl;
          std::vector<int64_t> prb(M, -1);
          int64_t pa = 0;
          for (int i = 0; i < M; ++i) {
            const int n = foff[i + 1] - foff[i];
            if (circh[i] && fhb[i] < 0) {
              prl.push_back(i);
              prb[i] = pa;
              pa += 4 * (int64_t)n;
            }
          }
          if (!prl.empty()) {
            h->npr = (int)prl.size();
            if ((st = upload(h, &h->pr_list, prl)) != PFMBEM_OK) return st;
            if ((st = upload(h, &h->pr_base, prb)) != PFMBEM_OK) return st;
            if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
            h->pr_val = dalloc<cplx>(h, (size_t)pa);
            h->pr_valf = dalloc<cplxf>(h, (size_t)pa);
            if (!h->pr_val || !h->pr_valf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (preconditioner)");
            CK(k_precond_rows(h));
          }
        }
      }
    }
  }
  if (!h->side) CK(pool_stream(h->dev, &h->side));
  if (!h->side_ev) CK(pool_event(h->dev, &h->side_ev));
  CK(cudaStreamWaitEvent(h->side, h->pre_ev, 0));
  h->astream = h->side;
  int64_t m2l_pairs = 0;
  m2l_lists.wait();
  for (int l = 1; l <= D; ++l) {
    Level& L = h->lev[l];
    M2LLists& o = m2l[l];
    L.nil = (int64_t)o.src.size();
    m2l_pairs += L.nil;
    pfmbem_status st;
    if ((st = upload(h, &L.il_ptr, o.ptr)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_src, o.src)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_off, o.off)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.il_img, o.img)) != PFMBEM_OK) return st;
    if (h->opt.m2l_mode == 2 || L.tc_fused) {
      L.tc_ntile = o.ntile;
      if ((st = upload(h, &L.tc_box, o.tbox)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.tc_noff, o.tnoff)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.tc_offs, o.toffs)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.tc_src, o.tsrc)) != PFMBEM_OK) return st;
      if ((st = upload(h, &L.tc_img, o.timg)) != PFMBEM_OK) return st;
    }
    L.nchunk = (int)o.cof.size();
    if ((st = upload(h, &L.pr_tgt, o.ptg)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.pr_src, o.psr)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.pr_img, o.pim)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.pr_off, o.pof)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.ch_off, o.cof)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.ch_beg, o.cbg)) != PFMBEM_OK) return st;
    if ((st = upload(h, &L.ch_end, o.cen)) != PFMBEM_OK) return st;
  }
  h->info.m2l_pairs = m2l_pairs;
  mark("M2L lists (overlapped)");
  if (cache && h->opt.launch == 0) {
    // top operators of the single-launch product, on the second stream once the
    // root operator (first set-up stream) and the M2M tables are there
    const size_t nrc = (size_t)NR * h->lev[0].P * 4 * NR * h->lev[1].P;   // [4 nr P1][nr P0]
    h->rootc = dalloc<cplx>(h, nrc);
    h->rootcf = dalloc<cplxf>(h, nrc);
    if (!h->rootc || !h->rootcf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (root operator)");
    if (D >= 3 && NR == 1) {
      const size_t P1 = h->lev[1].P, P3 = h->lev[3].P;
      h->m2m31 = dalloc<cplx>(h, 16 * P3 * P1);
      h->m2m31f = dalloc<cplxf>(h, 16 * P3 * P1);
      h->root1 = dalloc<cplx>(h, 16 * P1 * P1);
      h->root1f = dalloc<cplxf>(h, 16 * P1 * P1);
      if (!h->m2m31 || !h->m2m31f || !h->root1 || !h->root1f)
        return fail(h, PFMBEM_ENOMEM, "device allocation failed (top operators)");
    }
    if (h->aux[0]) CK(cudaStreamWaitEvent(h->side, h->aux_ev[0], 0));
    CK(k_top_operators(h, h->side));
    trace(h, h->side, "side: top operators done");
  }
  {
    pfmbem_status st;
    if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
  }
  mark("translation tables (overlapped)");
  // join: later work on the main stream sees every upload of the second stream
  CK(cudaEventRecord(h->side_ev, h->side));
  CK(cudaStreamWaitEvent(h->stream, h->side_ev, 0));
  for (int i = 0; i < 3; ++i)
    if (h->aux[i]) CK(cudaStreamWaitEvent(h->stream, h->aux_ev[i], 0));
  h->astream = nullptr;
  trace(h, h->stream, "main: streams joined");
  for (int l = 1; l <= D; ++l) {
    Level& L = h->lev[l];
    if (L.tc_B) CK(k_tc_build_operator(h, l));
    if (L.tc_Bf)
      CK(k_tc_build_operator_fused(h, l, 2 * (D >= 3 && NR == 1 ? std::min(L.p, std::max(1, L.p32)) : L.p) + 1));
  }
  if (cache) {
    // single-launch matvec unless the tensor-core M2L (its own kernel) is on
    bool tensor = false;
    for (int l = 1; l <= D; ++l) tensor = tensor || (h->lev[l].tc_B != nullptr && h->lev[l].tc_ntile > 0);
    if (h->opt.launch == 0 && !tensor) {
      pfmbem_status st;
      bool ok = false;
      if (!h->rootc) return fail(h, PFMBEM_ENOMEM, "single-launch product without its top operators");
      CK(k_fused_prepare(h, &ok));
      if (!ok && NR > 1) return fail(h, PFMBEM_EINVAL, "blocks wider than H need the single-launch product");
      if (ok) {
        std::vector<int> sli(E);
        {
          const Level& Lf = h->lev[D];
          for (size_t li = 0; li < Lf.hne.size(); ++li)
            for (int s2 = Lf.hbegin[Lf.hne[li]]; s2 < Lf.hend[Lf.hne[li]]; ++s2) sli[s2] = (int)li;
        }
        if ((st = upload(h, &h->s_li, sli)) != PFMBEM_OK) return st;
        // per sorted element, where its near-field row lies: (offset of the row's
        // blocks, first source << 32 | sources), one 16-byte load
        if (!nc_base.empty()) {
          std::vector<int64_t> meta(2 * (size_t)E, 0);
          const Level& Lf = h->lev[D];
          for (size_t li = 0; li < Lf.hne.size(); ++li) {
            const int b = Lf.hne[li], j0 = nc_sbase[li], ns = nc_sbase[li + 1] - j0;
            for (int s2 = Lf.hbegin[b]; s2 < Lf.hend[b]; ++s2) {
              meta[2 * (size_t)s2] = nc_base[li] + (int64_t)(s2 - Lf.hbegin[b]) * ns * 4;
              meta[2 * (size_t)s2 + 1] = ((int64_t)j0 << 32) | (int64_t)ns;
            }
          }
          if ((st = upload(h, &h->nr_meta, meta)) != PFMBEM_OK) return st;
          // the rows cut into pieces of at most 128 sources, each described in one
          // 16-byte load: offset of its first block (low, high word), its first
          // source in the concatenated list, (sources << 24) | element
          std::vector<int4> pieces;
          pieces.reserve((size_t)E + E / 2);
          for (int s2 = 0; s2 < E && E < (1 << 24); ++s2) {
            const int64_t r = meta[2 * (size_t)s2];
            const int j0 = (int)(meta[2 * (size_t)s2 + 1] >> 32), ns = (int)(meta[2 * (size_t)s2 + 1] & 0xffffffffll);
            for (int jb = 0; jb < std::max(ns, 1); jb += 128) {
              const int cnt = std::max(0, std::min(128, ns - jb));
              const uint64_t rp = (uint64_t)(r + 4 * (int64_t)jb);
              pieces.push_back(int4{(int)(uint32_t)(rp & 0xffffffffu), (int)(uint32_t)(rp >> 32), j0 + jb,
                                    (int)(((uint32_t)cnt << 24) | (uint32_t)s2)});
            }
          }
          h->nr_npiece = (int)pieces.size();
          if ((st = upload(h, &h->nr_piece, pieces)) != PFMBEM_OK) return st;
        }
        h->Un = dalloc<cplx>(h, (size_t)2 * E);
        h->Unf = dalloc<cplxf>(h, (size_t)2 * E);
        if (!h->Un || !h->Unf) return fail(h, PFMBEM_ENOMEM, "device allocation failed (near sums)");
        h->fz_bar = dalloc<unsigned long long>(h, 2);
        h->arn_bar = dalloc<unsigned long long>(h, 2);
        h->fz_err = dalloc<int>(h, 1);
        h->fz_stamp = dalloc<unsigned long long>(h, 32);
        // diagnostic: every block's arrival at every barrier (PFMBEM_BLOCK_TIMES)
        if (std::getenv("PFMBEM_BLOCK_TIMES")) h->fz_arrive = dalloc<unsigned long long>(h, (size_t)48 * 1024);
        if (!h->fz_bar || !h->arn_bar || !h->fz_err || !h->fz_stamp)
          return fail(h, PFMBEM_ENOMEM, "device allocation failed (barrier)");
        CK(cudaMemsetAsync(h->fz_bar, 0, 2 * sizeof(unsigned long long), h->stream));
        CK(cudaMemsetAsync(h->arn_bar, 0, 2 * sizeof(unsigned long long), h->stream));
        CK(cudaMemsetAsync(h->fz_err, 0, sizeof(int), h->stream));
        h->fused = true;
        h->pc = h->pc_val != nullptr || h->pr_val != nullptr;
        // the FP32 product's near sums in differences: lo parts of the densities and
        // the near blocks' FP64 row sums (built once the uploads below have landed)
        if (h->nc_vall) {
          h->fz_dlo = dalloc<cplxf>(h, 2 * (size_t)E);
          h->fz_rsum = dalloc<cplx>(h, 4 * (size_t)E);
          if (!h->fz_dlo || !h->fz_rsum) return fail(h, PFMBEM_ENOMEM, "device allocation failed (near row sums)");
        }
        // rows of the fibers applied by rows (not by FFT), for their FP64 row sums
        if (h->fz_nrowsum > 0 && h->fb_val) {
          h->fz_frs = dalloc<cplx>(h, 4 * (size_t)E);
          if (!h->fz_frs) return fail(h, PFMBEM_ENOMEM, "device allocation failed (fiber row sums)");
        }
      }
    }
  }
  mark("near + fiber integrals, P2M/L2P caches");
  {
    pfmbem_status st;
    if ((st = flush_uploads(h)) != PFMBEM_OK) return st;
  }
  h->ub_on = false;
  // tables of the single-launch product that read uploaded lists (s_li, the M2L pairs)
  if (h->fused) CK(k_fused_tables(h));
  // The create returns without waiting for the device: the caller's next work
  // queues behind the set-up on the same stream.  The operator check is read
  // back asynchronously and reported by the first call that waits
  // (check_ready).  With a timing mode on, the create waits here.
  if (h->trace_on || timing) {
    CK(cudaStreamSynchronize(h->stream));
    trace_report(h);
    mark("end of set-up");
  }
  pin_release_async(h);
  h->info.E = E;
  h->info.M = M;
  h->info.depth = D;
  h->info.nleaf_nonempty = h->lev[D].nne;
  h->info.p2m_nodes = h->g_far;
  h->info.lattice_q = h->lattice_q;
  h->info.root_x0 = h->x0;
  h->info.root_y0 = h->y0;
  h->info.nroot = h->nroot;
  h->info.super_p = h->nroot > 1 ? h->wide_ps : 0;
  h->setup_ms = now_ms() - t0;
  h->info.setup_ms = h->setup_ms;
  return PFMBEM_OK;
}

// ============================================================== staging
namespace {
struct InBuf {
  const cplx* dev = nullptr;
};
// Returns a device view of an input vector of n complex numbers.
pfmbem_status stage_input(pfmbem* h, const double* p, size_t n, cplx* scratch, const cplx** out) {
  if (is_device_ptr(p)) {
    *out = reinterpret_cast<const cplx*>(p);
    return PFMBEM_OK;
  }
  CK(cudaMemcpyAsync(scratch, p, n * sizeof(cplx), cudaMemcpyHostToDevice, h->stream));
  *out = scratch;
  return PFMBEM_OK;
}
}  // namespace

// ============================================================== GMRES
// Page-locked mirrors of the Arnoldi columns (2 (m + 2) complex numbers, m <= 250)
// are recycled between handles: allocating and freeing page-locked memory per
// solve costs more than the solve's host work.
namespace {
std::mutex g_small_mu;
std::vector<cplx*> g_small_free;
constexpr size_t kSmallPinned = sizeof(cplx) * 2 * (250 + 2);
}  // namespace

static cplx* pinned_small_get() {
  {
    std::lock_guard<std::mutex> lk(g_small_mu);
    if (!g_small_free.empty()) {
      cplx* p = g_small_free.back();
      g_small_free.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, kSmallPinned) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<cplx*>(p);
}

// The first call after create that waits for the handle's stream reports the
// set-up's operator check (non-finite M2L or root operator).
static pfmbem_status ready_checked(pfmbem* h) {
  if (h->ready) return PFMBEM_OK;
  h->ready = true;
  if (h->hstat && h->hstat[0])
    return fail(h, PFMBEM_ENUMERIC, "non-finite M2L operator; lower p or change depth");
  return PFMBEM_OK;
}

// Waits for the set-up of h once, then reports its operator check.
static pfmbem_status check_ready(pfmbem* h) {
  if (h->ready) return PFMBEM_OK;
  CK(cudaStreamSynchronize(h->stream));
  return ready_checked(h);
}

static void pinned_small_put(cplx* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_small_mu);
  g_small_free.push_back(p);
}

static pfmbem_status gmres_alloc(pfmbem* h, int m) {
  GmresWork& g = h->gw;
  const int n = 2 * h->E;
  if (g.V && g.m == m) return PFMBEM_OK;
  if (g.V) return PFMBEM_OK;   // keep the first allocation (restart length fixed per handle)
  g.n = n;
  g.m = m;
  g.V = dalloc<cplx>(h, (size_t)(m + 1) * n);
  g.w = dalloc<cplx>(h, n);
  g.r = dalloc<cplx>(h, n);
  g.x = dalloc<cplx>(h, n);
  g.b = dalloc<cplx>(h, n);
  g.d = dalloc<cplx>(h, n);
  g.c = dalloc<cplx>(h, n);
  g.hcol = dalloc<cplx>(h, 2 * (m + 2));
  g.nrm = dalloc<double>(h, 2);
  if (h->pc) g.Z = dalloc<cplx>(h, (size_t)m * n);
  if (!g.V || !g.w || !g.r || !g.x || !g.b || !g.d || !g.c || !g.hcol || !g.nrm || (h->pc && !g.Z))
    return fail(h, PFMBEM_ENOMEM, "GMRES workspace");
  if (h->arn_grid > 0) {
    g.H = dalloc<cplx>(h, (size_t)(m + 1) * m);
    g.cs = dalloc<cplx>(h, m);
    g.sn = dalloc<cplx>(h, m);
    g.gv = dalloc<cplx>(h, m + 1);
    g.acc = dalloc<cplx>(h, 2 * (2 * (size_t)(m + 1) + 1));
    g.y = dalloc<cplx>(h, m);
    g.ctl = dalloc<double>(h, 4);
    g.ictl = dalloc<int>(h, 4);
    if (!g.H || !g.cs || !g.sn || !g.gv || !g.acc || !g.y || !g.ctl || !g.ictl)
      return fail(h, PFMBEM_ENOMEM, "GMRES workspace");
  }
  g.hhost = pinned_small_get();
  if (!g.hhost) return fail(h, PFMBEM_ENOMEM, "pinned host buffer");
  return PFMBEM_OK;
}

static inline std::complex<double> toz(cplx a) { return {a.re, a.im}; }

// Estimate threshold (times tol) that ends an inner GMRES cycle of the refinement.
constexpr double kTrustThr = 0.5;

// Arnoldi steps enqueued per host check of the device-side GMRES cycle.
constexpr int kArnBatch = 4;

// One restart cycle of GMRES with the Arnoldi steps on the device (single-launch
// products): from V_0 = r / beta, the steps run as (preconditioner,) product
// and arnoldi step, kArnBatch at a time, and the host reads back only the done
// flag, the step count and the estimate after each batch.  Steps queued after
// the cycle finished return at once.  On return x += Z y (or V y), *steps and
// *est are the cycle's step count and residual estimate, *reason its end
// (1 estimate below thr, 2 breakdown, 3 restart length or maxit).
static pfmbem_status gmres_cycle_device(pfmbem* h, cplx* x, double beta, double bnorm, double thr, int max_steps,
                                        int precision, int* steps, double* est, int* reason) {
  GmresWork& g = h->gw;
  const int n = g.n, m = g.m;
  cplx* hh = g.hhost;
  double* hctl = reinterpret_cast<double*>(hh + 256);
  int* hictl = reinterpret_cast<int*>(hh + 260);
  CK(cudaMemsetAsync(g.gv, 0, sizeof(cplx) * (m + 1), h->stream));
  CK(cudaMemsetAsync(g.acc, 0, sizeof(cplx) * 2 * (2 * (size_t)(m + 1) + 1), h->stream));
  CK(cudaMemsetAsync(g.ictl, 0, sizeof(int) * 4, h->stream));
  hh[0] = cplx{beta, 0};
  hctl[0] = 1.0;
  hctl[1] = bnorm;
  hctl[2] = thr;
  CK(cudaMemcpyAsync(g.gv, hh, sizeof(cplx), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(g.ctl, hctl, 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  const int limit = std::min(m, max_steps);
  int j = 0, done_steps = 0;
  *reason = 0;
  // z_0 = P^-1 v_0 here; every later z_{j+1} comes out of the Arnoldi step j
  if (h->pc) CK(k_precond_apply(h, g.V, g.Z, precision));
  while (j < limit) {
    const int nb = std::min(kArnBatch, limit - j);
    for (int i = 0; i < nb; ++i, ++j) {
      const cplx* zj = (h->pc ? g.Z : g.V) + (size_t)j * n;
      CK(k_matvec_fused(h, zj, g.w, precision, g.ictl));
      CK(k_arnoldi_step(h, j, precision));
    }
    CK(cudaMemcpyAsync(hictl, g.ictl, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hctl + 3, g.ctl, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (h->fz_err) CK(cudaMemcpyAsync(hictl + 4, h->fz_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    done_steps = hictl[1];
    if (h->fz_err && hictl[4]) {
      // a bounded device-side wait gave up: the products and steps queued since
      // returned early, so the cycle stops here
      h->fz_dirty = true;
      return fail(h, PFMBEM_ETIMEOUT, "single-launch matvec: a bounded device-side wait gave up");
    }
    if (hictl[0]) {
      *reason = hictl[2];
      break;
    }
  }
  if (*reason == 0) *reason = 3;
  *steps = done_steps;
  *est = hctl[3];
  if (done_steps > 0) {
    CK(k_arnoldi_solve(h, g.y));
    CK(k_gemv_add(h, h->pc ? g.Z : g.V, done_steps, g.y, x, n));   // x += Z y (flexible) or V y
  }
  return PFMBEM_OK;
}

// A GMRES cycle ends once its Arnoldi residual estimate falls below f tol: f =
// 1/2 where the true residual is checked after the cycle (a margin against an
// optimistic estimate); for the inner solves of the refinement, which trust the
// estimate and whose error the FP64 residual of the next refinement step
// corrects, f = trust_thr() (PFMBEM_INNER_THR overrides, for measurement).
static double trust_thr() {
  static const double f = [] {
    const char* v = std::getenv("PFMBEM_INNER_THR");
    return v ? std::atof(v) : kTrustThr;
  }();
  return f;
}

// Restarted GMRES(m) with classical Gram-Schmidt applied twice; A is applied by
// the FMM matvec in the given precision.  Solves A x = b in place of x (device).
// Restarted GMRES(m) with CGS2 Arnoldi, flexibly right-preconditioned by the
// fibers' inverse same-fiber blocks when the handle has them (Sec. 4 solves
// with a preconditioned GMRES; this is the block-Jacobi choice).  With
// trust_estimate the solve ends as
// soon as the Arnoldi residual estimate falls below tol/2, without recomputing
// the true residual (inner solves of the refinement, whose outer loop computes
// the FP64 residual anyway).  A caller that already holds ||b|| passes it as
// known_bnorm (> 0), which saves a device-to-host round trip; on a zero start
// the first residual is b itself and its norm is not recomputed either.
static pfmbem_status gmres(pfmbem* h, const cplx* b, cplx* x, double tol, int maxit, int precision,
                           int* iters_out, int* restarts_out, double* relres_out, bool zero_start = false,
                           bool trust_estimate = false, double known_bnorm = 0) {
  GmresWork& g = h->gw;
  const int n = g.n, m = g.m;
  double* hn = reinterpret_cast<double*>(g.hhost);
  double bnorm = known_bnorm;
  if (!(bnorm > 0)) {
    CK(k_norm2(h, b, n, g.nrm));
    CK(cudaMemcpyAsync(hn, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    bnorm = std::sqrt(hn[0]);
  }
  if (bnorm == 0) {
    CK(cudaMemsetAsync(x, 0, sizeof(cplx) * n, h->stream));
    *iters_out = 0;
    *relres_out = 0;
    return PFMBEM_OK;
  }
  int iters = 0, restarts = 0;
  double relres = 1.0;
  bool done = false;
  std::vector<std::complex<double>> Hm((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1);
  while (!done) {
    // r = b - A x (x = 0 on a zero start)
    double beta = bnorm;
    if (zero_start && restarts == 0) {
      CK(cudaMemcpyAsync(g.r, b, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CK(k_matvec(h, x, g.w, precision));
      CK(k_sub(h, b, g.w, g.r, n));
      CK(k_norm2(h, g.r, n, g.nrm));
      CK(cudaMemcpyAsync(hn, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      beta = std::sqrt(hn[0]);
    }
    relres = beta / bnorm;
    if (!std::isfinite(relres)) return fail(h, PFMBEM_ENUMERIC, "non-finite residual");
    if (relres <= tol || iters >= maxit) break;
    CK(k_scale_copy(h, g.r, cplx{1.0 / beta, 0}, g.V, n));
    if (h->arn_grid > 0 && h->fused && h->cached && m < 256) {
      int steps = 0, reason = 0;
      double est = 1;
      pfmbem_status sc = gmres_cycle_device(h, x, beta, bnorm, (trust_estimate ? trust_thr() : 0.5) * tol,
                                            maxit - iters, precision, &steps, &est, &reason);
      if (sc != PFMBEM_OK) return sc;
      iters += steps;
      ++restarts;
      if (steps == 0) break;            // no progress (the cycle stopped at once): leave with the current residual
      if (reason != 3 && trust_estimate) {
        relres = est;
        done = true;
      }
      continue;
    }
    std::fill(gvec.begin(), gvec.end(), 0.0);
    gvec[0] = beta;
    int j = 0;
    for (; j < m && iters < maxit; ++j) {
      cplx* vj = g.V + (size_t)j * n;
      cplx* vj1 = g.V + (size_t)(j + 1) * n;
      if (h->pc) {
        // flexible right preconditioning: z_j = P^-1 v_j, w = A z_j
        cplx* zj = g.Z + (size_t)j * n;
        CK(k_precond_apply(h, vj, zj, precision));
        CK(k_matvec(h, zj, g.w, precision));
      } else {
        CK(k_matvec(h, vj, g.w, precision));
      }
      ++iters;
      // CGS2
      CK(k_multidot(h, g.V, j + 1, g.w, n, g.hcol));
      CK(k_gemv_sub(h, g.V, j + 1, g.hcol, g.w, n));
      CK(k_multidot(h, g.V, j + 1, g.w, n, g.hcol + (m + 2)));
      CK(k_gemv_sub(h, g.V, j + 1, g.hcol + (m + 2), g.w, n));
      CK(k_norm2(h, g.w, n, g.nrm));
      CK(cudaMemcpyAsync(g.hhost, g.hcol, sizeof(cplx) * 2 * (m + 2), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(hn + 4 * (m + 2) - 2, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      double hnext = std::sqrt(hn[4 * (m + 2) - 2]);
      for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = toz(g.hhost[i]) + toz(g.hhost[(m + 2) + i]);
      Hm[(size_t)(j + 1) * m + j] = hnext;
      if (hnext > 0) CK(k_scale_copy(h, g.w, cplx{1.0 / hnext, 0}, vj1, n));
      // Givens
      for (int i = 0; i < j; ++i) {
        auto a = Hm[(size_t)i * m + j], bb = Hm[(size_t)(i + 1) * m + j];
        Hm[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
        Hm[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      auto a = Hm[(size_t)j * m + j], bb = Hm[(size_t)(j + 1) * m + j];
      double den = std::sqrt(std::norm(a) + std::norm(bb));
      if (den == 0) { cs[j] = 1; sn[j] = 0; }
      else { cs[j] = a / den; sn[j] = bb / den; }
      Hm[(size_t)j * m + j] = std::conj(cs[j]) * a + std::conj(sn[j]) * bb;
      Hm[(size_t)(j + 1) * m + j] = 0;
      auto gj = gvec[j];
      gvec[j] = std::conj(cs[j]) * gj;
      gvec[j + 1] = -sn[j] * gj;
      double est = std::abs(gvec[j + 1]) / bnorm;
      if (est <= (trust_estimate ? trust_thr() : 0.5) * tol || hnext == 0) {
        ++j;
        if (trust_estimate) {
          relres = est;
          done = true;
        }
        break;
      }
    }
    // back substitution and x += V y
    std::vector<std::complex<double>> y(j);
    for (int i = j - 1; i >= 0; --i) {
      auto s = gvec[i];
      for (int q = i + 1; q < j; ++q) s -= Hm[(size_t)i * m + q] * y[q];
      y[i] = s / Hm[(size_t)i * m + i];
    }
    for (int i = 0; i < j; ++i) g.hhost[i] = cplx{y[i].real(), y[i].imag()};
    CK(cudaMemcpyAsync(g.hcol, g.hhost, sizeof(cplx) * j, cudaMemcpyHostToDevice, h->stream));
    CK(k_gemv_add(h, h->pc ? g.Z : g.V, j, g.hcol, x, n));   // x += Z y (flexible) or V y
    ++restarts;
  }
  *iters_out = iters;
  *restarts_out = restarts;
  *relres_out = relres;
  return relres <= tol ? PFMBEM_OK : PFMBEM_ENOCONV;
}

// ============================================================== batched solve
// Blocks per instance group of the persistent batched launch.
constexpr int kBatchGroup = 8;

// Lockstep iterative refinement over many handles: every instance is a small
// state machine (outer FP64 residual, then Arnoldi steps of an inner GMRES on
// the handle's operator precision); each lockstep phase enqueues one unit of
// work per active instance on that instance's stream, then waits once for all.
namespace {
enum BState { B_RESID, B_ARNOLDI, B_DONE };
struct BInst {
  pfmbem* h = nullptr;
  BState state = B_RESID;
  int prec = PFMBEM_FP64;
  double bn = 0, relres = 1, prev = 1e300, inner_tol = 1e-4, beta = 0;
  int iters = 0, refinements = 0, stalls = 0, j = 0;
  bool zero_x = true;
  pfmbem_status st = PFMBEM_ENOCONV;
  std::vector<std::complex<double>> Hm, cs, sn, gv;
  double t0 = 0;
};
}  // namespace

static pfmbem_status batch_enqueue(BInst& b) {
  pfmbem* h = b.h;
  GmresWork& g = h->gw;
  const int n = g.n, m = g.m;
  if (b.state == B_RESID) {
    if (b.zero_x) {
      CK(cudaMemcpyAsync(g.d, g.b, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CK(k_matvec(h, g.x, g.w, PFMBEM_FP64));
      CK(k_sub(h, g.b, g.w, g.d, n));
    }
    CK(k_norm2(h, g.d, n, g.nrm));
    CK(cudaMemcpyAsync(g.hhost, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  } else if (b.state == B_ARNOLDI) {
    cplx* vj = g.V + (size_t)b.j * n;
    if (h->pc) {
      // flexible right preconditioning, as in the single solve
      cplx* zj = g.Z + (size_t)b.j * n;
      CK(k_precond_apply(h, vj, zj, b.prec));
      CK(k_matvec(h, zj, g.w, b.prec));
    } else {
      CK(k_matvec(h, vj, g.w, b.prec));
    }
    CK(k_multidot(h, g.V, b.j + 1, g.w, n, g.hcol));
    CK(k_gemv_sub(h, g.V, b.j + 1, g.hcol, g.w, n));
    CK(k_multidot(h, g.V, b.j + 1, g.w, n, g.hcol + (m + 2)));
    CK(k_gemv_sub(h, g.V, b.j + 1, g.hcol + (m + 2), g.w, n));
    CK(k_norm2(h, g.w, n, g.nrm));
    CK(cudaMemcpyAsync(g.hhost, g.hcol, sizeof(cplx) * 2 * (m + 2), cudaMemcpyDeviceToHost, h->stream));
    double* hn = reinterpret_cast<double*>(g.hhost);
    CK(cudaMemcpyAsync(hn + 4 * (m + 2) - 2, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  return PFMBEM_OK;
}

// Finish the inner GMRES of instance b: x += V y; next is the FP64 residual.
static pfmbem_status batch_finish_inner(BInst& b) {
  pfmbem* h = b.h;
  GmresWork& g = h->gw;
  const int m = g.m, j = b.j;
  std::vector<std::complex<double>> y(j);
  for (int i = j - 1; i >= 0; --i) {
    auto s = b.gv[i];
    for (int q = i + 1; q < j; ++q) s -= b.Hm[(size_t)i * m + q] * y[q];
    y[i] = s / b.Hm[(size_t)i * m + i];
  }
  // the pinned mirror is free again: this instance's stream has synchronised
  for (int i = 0; i < j; ++i) g.hhost[i] = cplx{y[i].real(), y[i].imag()};
  CK(cudaMemcpyAsync(g.hcol, g.hhost, sizeof(cplx) * j, cudaMemcpyHostToDevice, h->stream));
  CK(k_gemv_add(h, h->pc ? g.Z : g.V, j, g.hcol, g.x, g.n));
  b.zero_x = false;
  b.state = B_RESID;
  return PFMBEM_OK;
}

// Host processing after the lockstep wait.
static pfmbem_status batch_advance(BInst& b, double tol, int maxit) {
  pfmbem* h = b.h;
  GmresWork& g = h->gw;
  const int n = g.n, m = g.m;
  double* hn = reinterpret_cast<double*>(g.hhost);
  if (b.state == B_RESID) {
    const double rn = std::sqrt(hn[0]);
    if (b.refinements == 0 && b.zero_x) b.bn = rn;
    b.relres = b.bn > 0 ? rn / b.bn : 0.0;
    if (!std::isfinite(b.relres)) { b.st = PFMBEM_ENUMERIC; b.state = B_DONE; return PFMBEM_OK; }
    if (b.relres <= tol) { b.st = PFMBEM_OK; b.state = B_DONE; return PFMBEM_OK; }
    if (b.iters >= maxit || b.refinements >= 50) { b.st = PFMBEM_ENOCONV; b.state = B_DONE; return PFMBEM_OK; }
    if (b.relres > 0.5 * b.prev) {
      if (++b.stalls >= 3) { b.st = PFMBEM_ENOCONV; b.state = B_DONE; return PFMBEM_OK; }
    } else {
      b.stalls = 0;
    }
    b.prev = b.relres;
    b.refinements++;
    // start an inner GMRES on d with V_0 = d / ||d||
    b.inner_tol = b.prec == PFMBEM_MIXED ? std::max(1e-4, 0.3 * tol / b.relres) : 0.5 * tol / b.relres;
    b.beta = rn;
    b.j = 0;
    std::fill(b.gv.begin(), b.gv.end(), 0.0);
    b.gv[0] = rn;
    CK(k_scale_copy(h, g.d, cplx{1.0 / rn, 0}, g.V, n));
    b.state = B_ARNOLDI;
    return PFMBEM_OK;
  }
  if (b.state == B_ARNOLDI) {
    const int j = b.j;
    const double hnext = std::sqrt(hn[4 * (m + 2) - 2]);
    for (int i = 0; i <= j; ++i) b.Hm[(size_t)i * m + j] = toz(g.hhost[i]) + toz(g.hhost[(m + 2) + i]);
    b.Hm[(size_t)(j + 1) * m + j] = hnext;
    if (hnext > 0) CK(k_scale_copy(h, g.w, cplx{1.0 / hnext, 0}, g.V + (size_t)(j + 1) * n, n));
    for (int i = 0; i < j; ++i) {
      auto a = b.Hm[(size_t)i * m + j], bb = b.Hm[(size_t)(i + 1) * m + j];
      b.Hm[(size_t)i * m + j] = std::conj(b.cs[i]) * a + std::conj(b.sn[i]) * bb;
      b.Hm[(size_t)(i + 1) * m + j] = -b.sn[i] * a + b.cs[i] * bb;
    }
    auto a = b.Hm[(size_t)j * m + j], bb = b.Hm[(size_t)(j + 1) * m + j];
    const double den = std::sqrt(std::norm(a) + std::norm(bb));
    if (den == 0) { b.cs[j] = 1; b.sn[j] = 0; }
    else { b.cs[j] = a / den; b.sn[j] = bb / den; }
    b.Hm[(size_t)j * m + j] = std::conj(b.cs[j]) * a + std::conj(b.sn[j]) * bb;
    b.Hm[(size_t)(j + 1) * m + j] = 0;
    const auto gj = b.gv[j];
    b.gv[j] = std::conj(b.cs[j]) * gj;
    b.gv[j + 1] = -b.sn[j] * gj;
    b.iters++;
    b.j = j + 1;
    const double est = std::abs(b.gv[j + 1]) / b.beta;
    if (est <= b.inner_tol || hnext == 0 || b.j >= m || b.iters >= maxit) return batch_finish_inner(b);
  }
  return PFMBEM_OK;
}

// ============================================================== C ABI
extern "C" {

pfmbem_status pfmbem_solve_batch(int ninst, const pfmbem_t* hs, double* const* psis, int use_guess, double tol,
                                 int maxit, pfmbem_info* infos) {
  if (ninst < 0 || (ninst > 0 && (!hs || !psis)) || !(tol > 0) || maxit < 1) return PFMBEM_EINVAL;
  for (int i = 0; i < ninst; ++i)
    if (hs[i] && !hs[i]->ready) {
      const pfmbem_status rs = check_ready(hs[i]);
      if (rs != PFMBEM_OK) return rs;
    }
  std::vector<BInst> inst(ninst);
  const double t0 = now_ms();
  for (int i = 0; i < ninst; ++i) {
    pfmbem* h = hs[i];
    if (!h || !psis[i]) return PFMBEM_EINVAL;
    if (h->tree == 1) return fail(h, PFMBEM_EINVAL, "the batched solver takes square-tree handles only");
    BInst& b = inst[i];
    b.h = h;
    b.prec = (h->opt.precision == PFMBEM_MIXED && h->cached) ? PFMBEM_MIXED : PFMBEM_FP64;
    const int m = h->opt.gmres_m > 0 ? h->opt.gmres_m : 60;
    if (m > 250) return fail(h, PFMBEM_EINVAL, "gmres_m above 250");
    pfmbem_status st = gmres_alloc(h, m);
    if (st != PFMBEM_OK) return st;
    GmresWork& g = h->gw;
    b.Hm.assign((size_t)(g.m + 1) * g.m, 0.0);
    b.cs.assign(g.m, 0.0);
    b.sn.assign(g.m, 0.0);
    b.gv.assign(g.m + 1, 0.0);
    CK(k_rhs(h, g.b));
    if (use_guess) {
      // the initial guess, from host or device memory
      CK(cudaMemcpyAsync(g.x, psis[i], sizeof(cplx) * g.n,
                         is_device_ptr(psis[i]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
      b.zero_x = false;
      // ||b|| for the lockstep's relative residuals (the persistent launch forms its own)
      double bn2 = 0;
      CK(k_norm2(h, g.b, g.n, g.nrm));
      CK(cudaMemcpyAsync(&bn2, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      b.bn = std::sqrt(bn2);
    } else {
      CK(cudaMemsetAsync(g.x, 0, sizeof(cplx) * g.n, h->stream));
    }
  }
  // One persistent launch over all instances when every handle can run in it
  // (PFMBEM_BATCH_LOCKSTEP=1 keeps the host-driven lockstep below, for
  // measurement); PFMBEM_BATCH_GROUP sets the blocks per instance group.
  static const bool lockstep = std::getenv("PFMBEM_BATCH_LOCKSTEP") != nullptr;
  bool persist = !lockstep && ninst > 0;
  for (int i = 0; persist && i < ninst; ++i) persist = batch_eligible(hs[i]);
  if (persist) {
    static const char* gsenv = std::getenv("PFMBEM_BATCH_GROUP");
    int GS = 0;
    for (int i = 0; i < ninst; ++i) GS = std::max(GS, hs[i]->opt.batch_group);
    if (GS <= 0) GS = kBatchGroup;
    if (gsenv) GS = std::max(1, std::atoi(gsenv));
    // longest first (LPT): the instances by element count, descending
    std::vector<int> order(ninst);
    for (int i = 0; i < ninst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->E > hs[b]->E; });
    pfmbem* h = hs[0];                 // errors are reported on the first handle
    cudaStream_t st = h->stream;
    // the launch runs on the first handle's stream, after every handle's
    // pending work (set-up tails, right-hand sides)
    std::vector<BatchResult> res(ninst);
    int timed_out = 0;
    const cudaError_t e = k_batch_solve(ninst, hs, order.data(), GS, tol, maxit, trust_thr(), use_guess, st,
                                        res.data(), &timed_out);
    if (e == cudaErrorNotSupported) {
      cudaGetLastError();
      persist = false;                 // the lockstep below
    } else if (e != cudaSuccess) {
      return fail_cuda(h, e, "batched solve");
    } else {
      pfmbem_status worst = PFMBEM_OK;
      for (int i = 0; i < ninst; ++i) {
        const bool pdev = is_device_ptr(psis[i]);
        CK(cudaMemcpyAsync(psis[i], hs[i]->gw.x, sizeof(cplx) * hs[i]->gw.n,
                           pdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
      }
      CK(cudaStreamSynchronize(st));
      const double ms = now_ms() - t0;
      for (int i = 0; i < ninst; ++i) {
        pfmbem_status si = timed_out ? PFMBEM_ETIMEOUT : (pfmbem_status)res[i].status;
        if (timed_out) hs[i]->err = "batched solve: a bounded device-side wait gave up";
        if (infos) {
          infos[i].iters = res[i].iters;
          infos[i].restarts = res[i].refinements;
          infos[i].rel_residual = res[i].relres;
          infos[i].ms = ms;
          infos[i].status = si;
        }
        if (si != PFMBEM_OK && worst == PFMBEM_OK) worst = si;
      }
      return worst;
    }
  }
  int active = ninst;
  while (active > 0) {
    for (auto& b : inst)
      if (b.state != B_DONE) {
        pfmbem_status st = batch_enqueue(b);
        if (st != PFMBEM_OK) return st;
      }
    for (auto& b : inst)
      if (b.state != B_DONE) {
        pfmbem* h = b.h;
        CK(cudaStreamSynchronize(h->stream));
      }
    active = 0;
    for (auto& b : inst) {
      if (b.state == B_DONE) continue;
      pfmbem_status st = batch_advance(b, tol, maxit);
      if (st != PFMBEM_OK) return st;
      if (b.state != B_DONE) ++active;
    }
  }
  pfmbem_status worst = PFMBEM_OK;
  for (int i = 0; i < ninst; ++i) {
    BInst& b = inst[i];
    pfmbem* h = b.h;
    GmresWork& g = h->gw;
    const bool pdev = is_device_ptr(psis[i]);
    CK(cudaMemcpyAsync(psis[i], g.x, sizeof(cplx) * g.n, pdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
  }
  for (int i = 0; i < ninst; ++i) {
    BInst& b = inst[i];
    pfmbem* h = b.h;
    CK(cudaStreamSynchronize(h->stream));
    if (infos) {
      infos[i].iters = b.iters;
      infos[i].restarts = b.refinements;
      infos[i].rel_residual = b.relres;
      infos[i].ms = now_ms() - t0;
      infos[i].status = b.st;
    }
    if (b.st != PFMBEM_OK && worst == PFMBEM_OK) worst = b.st;
  }
  return worst;
}

pfmbem_status pfmbem_create(int M, const int* nodes_per_fiber, const double* nodes_xy, double H, int lattice,
                            double k, double k1, double rho_ratio, double theta, const pfmbem_options* opt,
                            void* cuda_stream, pfmbem_t* out) {
  if (!out) return PFMBEM_EINVAL;
  *out = nullptr;
  if (M < 1 || !nodes_per_fiber || !nodes_xy) return PFMBEM_EINVAL;
  if (!(H > 0) || !(k > 0) || !(k1 > 0) || !(rho_ratio > 0) || !std::isfinite(theta)) return PFMBEM_EINVAL;
  pfmbem* h = new pfmbem();
  h->M = M;
  h->H = H;
  h->lattice = lattice;
  h->k = k;
  h->k1 = k1;
  h->rho = rho_ratio;
  h->theta = theta;
  if (opt) h->opt = *opt;
  h->eta = h->opt.eta != 0 ? h->opt.eta : k;
  h->beta = k * H * std::sin(theta);
  h->alpha = cplx{std::cos(h->beta), std::sin(h->beta)};
  {
    // c2 = 2 / (i eta (1 + rho)) = -2i / (eta (1 + rho))
    h->c2re = 0.0;
    h->c2im = -2.0 / (h->eta * (1.0 + rho_ratio));
  }
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  // Wood anomalies (Sec. 2): kH(1 +- sin theta) = 2 pi n
  {
    double s = std::sin(theta), dmin = 1e300;
    for (double v : {k * H * (1 + s), k * H * (1 - s)}) {
      double r = v - 2 * M_PI * std::round(v / (2 * M_PI));
      dmin = std::min(dmin, std::fabs(r));
    }
    if (dmin < 1e-3) {
      h->err = "incidence within 1e-3 of a Wood anomaly";
      *out = h;
      return PFMBEM_EWOOD;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    h->err = "no CUDA device";
    *out = h;
    return PFMBEM_ECUDA;
  }
  ensure_gauss();
  ensure_pool();
  cudaGetDevice(&h->dev);
  h->prof.on = h->opt.profile != 0;
  // host copies of the inputs
  std::vector<int> npf(M);
  if (is_device_ptr(nodes_per_fiber)) {
    if (cudaMemcpy(npf.data(), nodes_per_fiber, sizeof(int) * M, cudaMemcpyDeviceToHost) != cudaSuccess) {
      *out = h;
      return fail_cuda(h, cudaGetLastError(), "copy nodes_per_fiber");
    }
  } else {
    std::memcpy(npf.data(), nodes_per_fiber, sizeof(int) * M);
  }
  long long tot = 0;
  for (int i = 0; i < M; ++i) tot += npf[i] > 0 ? npf[i] : 0;
  std::vector<double> nodes(2 * tot);
  if (is_device_ptr(nodes_xy)) {
    if (cudaMemcpy(nodes.data(), nodes_xy, sizeof(double) * 2 * tot, cudaMemcpyDeviceToHost) != cudaSuccess) {
      *out = h;
      return fail_cuda(h, cudaGetLastError(), "copy nodes");
    }
  } else {
    std::memcpy(nodes.data(), nodes_xy, sizeof(double) * 2 * tot);
  }
  *out = h;
  pfmbem_status st = build_plan(h, npf.data(), nodes.data());
  if (st != PFMBEM_OK) return st;
  h->hstat = reinterpret_cast<int*>(pinned_small_get());
  if (!h->hstat) return fail(h, PFMBEM_ENOMEM, "pinned host buffer");
  h->hstat[0] = 0;
  CK(cudaMemcpyAsync(h->hstat, h->tab_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  h->ready = false;
  return PFMBEM_OK;
}


void pfmbem_destroy(pfmbem_t h) {
  if (!h) return;
  if (h->side) cudaStreamSynchronize(h->side);
  for (int i = 0; i < 3; ++i)
    if (h->aux[i]) cudaStreamSynchronize(h->aux[i]);
  for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  pin_release(h);                  // a create that failed part-way
  pinned_small_put(h->gw.hhost);
  pinned_small_put(reinterpret_cast<cplx*>(h->hstat));
  pool_put(h->dev, h->side_ev);
  pool_put(h->dev, h->pre_ev);
  pool_put(h->dev, h->side);
  for (int i = 0; i < 3; ++i) {
    pool_put(h->dev, h->aux_ev[i]);
    pool_put(h->dev, h->aux[i], i == 2);
  }
  pool_put(h->dev, h->fork_ev);
  pool_put(h->dev, h->ktab_ev);
  prof_release(h);
  for (cudaEvent_t e : h->trace_ev) cudaEventDestroy(e);
  delete h;
}

const char* pfmbem_last_error(pfmbem_t h) { return h ? h->err.c_str() : "null handle"; }

pfmbem_status pfmbem_plan(pfmbem_t h, pfmbem_plan_info* info) {
  if (!h || !info) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  if ((h->cached || h->tri_cache) && h->stat_dev) {
    unsigned long long c[4];
    CK(cudaMemcpyAsync(c, h->stat_dev, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->info.near_pairs = (int64_t)c[0];
    h->info.near_quad = (int64_t)c[1];
    h->info.fiber_pairs = (int64_t)c[2];
    h->info.fiber_quad = (int64_t)c[3];
  }
  h->info.cached = h->cached ? 1 : 0;
  h->info.tc_levels = h->fused ? k_fused_tc_levels(h) : 0;
  for (int l = 0; l < 16; ++l) {
    h->info.p32[l] = l <= h->D ? (h->fused ? (k_fused_order(h, l, true) - 1) / 2 : h->lev[l].p) : 0;
    h->info.m2l_pairs_level[l] = l <= h->D ? (int64_t)h->lev[l].nil : 0;
  }
  h->info.near_blocks = h->cached || h->tri_cache ? h->nc_blocks : 0;
  h->info.fiber_entries = h->cached || h->tri_cache ? h->fb_entries : 0;
  *info = h->info;
  return PFMBEM_OK;
}

pfmbem_status pfmbem_rhs(pfmbem_t h, double* B) {
  if (!h || !B) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t n = 2 * (size_t)h->E;
  if (is_device_ptr(B)) {
    CK(k_rhs(h, reinterpret_cast<cplx*>(B)));
    return PFMBEM_OK;
  }
  CK(k_rhs(h, h->stage_out));
  CK(cudaMemcpyAsync(B, h->stage_out, n * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PFMBEM_OK;
}

pfmbem_status pfmbem_matvec(pfmbem_t h, const double* x, double* y, int precision) {
  if (!h || !x || !y) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  if (precision != PFMBEM_FP64 && precision != PFMBEM_MIXED) return fail(h, PFMBEM_EINVAL, "precision");
  const size_t n = 2 * (size_t)h->E;
  const cplx* xd;
  pfmbem_status st = stage_input(h, x, n, h->stage_in, &xd);
  if (st != PFMBEM_OK) return st;
  const bool ydev = is_device_ptr(y);
  cplx* yd = ydev ? reinterpret_cast<cplx*>(y) : h->stage_out;
  CK(k_matvec(h, xd, yd, precision));
  if (!ydev) {
    // a host result waits for the product, so a device-side wait that gave up is reported here
    int fze = 0;
    CK(cudaMemcpyAsync(y, yd, n * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
    if (h->fused && h->fz_err && h->hstat) {
      h->hstat[2] = 0;
      CK(cudaMemcpyAsync(h->hstat + 2, h->fz_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (h->fused && h->fz_err && h->hstat) fze = h->hstat[2];
    if (fze) {
      h->fz_dirty = true;
      return fail(h, PFMBEM_ETIMEOUT, "single-launch matvec: a bounded device-side wait gave up");
    }
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_solve(pfmbem_t h, const double* B, double* psi, int use_guess, double tol, int maxit,
                           pfmbem_info* info) {
  if (!h || !psi || !(tol > 0) || maxit < 1) return PFMBEM_EINVAL;
  const double t0 = now_ms();
  const int m = h->opt.gmres_m > 0 ? h->opt.gmres_m : 60;
  if (m > 250) return fail(h, PFMBEM_EINVAL, "gmres_m above 250");
  pfmbem_status st = gmres_alloc(h, m);
  if (st != PFMBEM_OK) return st;
  GmresWork& g = h->gw;
  const size_t n = 2 * (size_t)h->E;
  if (B) {
    const cplx* bd;
    if ((st = stage_input(h, B, n, g.b, &bd)) != PFMBEM_OK) return st;
    if (bd != g.b) CK(cudaMemcpyAsync(g.b, bd, n * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    CK(k_rhs(h, g.b));
  }
  const bool pdev = is_device_ptr(psi);
  if (use_guess) {
    CK(cudaMemcpyAsync(g.x, psi, n * sizeof(cplx), pdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  } else {
    CK(cudaMemsetAsync(g.x, 0, n * sizeof(cplx), h->stream));
  }
  int iters = 0, restarts = 0;
  double relres = 1;
  bool guess32 = false;
  if (use_guess) {
    // Scale the guess x by the gamma minimising ||B - gamma A x|| (w = A x from
    // one FP64 matvec, gamma = <w, B> / <w, w>); the scaled guess is kept when
    // its residual d = B - gamma w is below ||B||, else the solve starts at zero.
    // (mixed precision: A x is the FP32 product; its residual only starts the
    // refinement, and convergence is decided on FP64 residuals)
    double nn[2] = {0, 0}, rn = 0;
    cplx wb{0, 0};
    guess32 = h->opt.precision == PFMBEM_MIXED && h->cached && h->fused;
    CK(k_matvec(h, g.x, g.w, guess32 ? PFMBEM_MIXED : PFMBEM_FP64));
    CK(k_norm2(h, g.b, (int)n, g.nrm));
    CK(k_norm2(h, g.w, (int)n, g.nrm + 1));
    CK(k_multidot(h, g.w, 1, g.b, (int)n, g.hcol));
    CK(cudaMemcpyAsync(nn, g.nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&wb, g.hcol, sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const cplx gam = nn[1] > 0 ? cplx{wb.re / nn[1], wb.im / nn[1]} : cplx{0, 0};
    CK(k_scale_copy(h, g.x, gam, g.c, (int)n));
    CK(cudaMemcpyAsync(g.x, g.c, n * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(g.d, g.b, n * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
    CK(k_axpy(h, cplx{-gam.re, -gam.im}, g.w, g.d, (int)n));
    CK(k_norm2(h, g.d, (int)n, g.nrm));
    CK(cudaMemcpyAsync(&rn, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!(rn < nn[0])) {
      CK(cudaMemsetAsync(g.x, 0, n * sizeof(cplx), h->stream));
      use_guess = 0;
    }
  }
  if (h->opt.precision == PFMBEM_MIXED && h->cached) {
    // FP64 iterative refinement: r = B - A x with the FP64 operator, an inner
    // GMRES on the mixed-precision operator solves A d = r loosely, x += d.
    double bn = 0;
    {
      CK(k_norm2(h, g.b, (int)n, g.nrm));
      CK(cudaMemcpyAsync(&bn, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      bn = std::sqrt(bn);
    }
    st = PFMBEM_ENOCONV;
    int refinements = 0, stalls = 0;
    double prev = 1e300;
    // (PFMBEM_R1_FP64=1 computes every refinement residual in FP64, for measurement)
    static const bool r1_fp64 = std::getenv("PFMBEM_R1_FP64") != nullptr;
    const bool fast_r1 = !r1_fp64 && h->fused;
    for (; refinements < 50; ++refinements) {
      // The second residual comes from the FP32 product: its error on smooth
      // densities (~2e-7 of ||B||) lies below what that step asks of its inner
      // solve, and the FP64 residual of the following step is the check, so no
      // convergence is declared on it.  One FP64 product per solve fewer.
      const bool r32 = refinements == 1 && fast_r1;
      if (refinements == 0 && !use_guess) {
        // x = 0: the residual is B itself
        CK(cudaMemcpyAsync(g.d, g.b, n * sizeof(cplx), cudaMemcpyDeviceToDevice, h->stream));
      } else if (refinements == 0) {
        // the scaled guess: d = B - gamma A x is already in place
      } else {
        CK(k_matvec(h, g.x, g.w, r32 ? PFMBEM_MIXED : PFMBEM_FP64));
        CK(k_sub(h, g.b, g.w, g.d, (int)n));
      }
      double rn = bn * bn;             // d = B at a zero start
      if (refinements > 0 || use_guess) {
        CK(k_norm2(h, g.d, (int)n, g.nrm));
        CK(cudaMemcpyAsync(&rn, g.nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
      }
      relres = bn > 0 ? std::sqrt(rn) / bn : 0.0;
      if (!std::isfinite(relres)) return fail(h, PFMBEM_ENUMERIC, "non-finite residual");
      if (relres <= tol && !r32 && !(refinements == 0 && guess32 && use_guess)) { st = PFMBEM_OK; break; }
      if (iters >= maxit) break;
      // stop when refinement no longer reduces the FP64 residual
      if (!r32) {
        if (relres > 0.5 * prev) { if (++stalls >= 3) break; } else stalls = 0;
        prev = relres;
      }
      // The FP32 operator puts a floor of roughly eps_32 * cond under the inner
      // residual, so the inner solve is asked for a modest reduction and its
      // work per refinement step is bounded; refinement does the rest.  The
      // first step aims at an absolute residual of 1e-4 ||B|| (a guess that
      // already sits below ||B|| needs a smaller relative reduction), later
      // steps at 0.3 tol ||B||.
      const double target = refinements == 0 ? std::max(1e-4, 0.3 * tol) : 0.3 * tol;
      const double inner_tol = std::max(1e-4, std::min(0.5, target / relres));
      const int cap = std::min(maxit - iters, 4 * g.m);
      int it = 0, rs = 0;
      double rr = 1;
      CK(cudaMemsetAsync(g.c, 0, n * sizeof(cplx), h->stream));
      pfmbem_status si = gmres(h, g.d, g.c, inner_tol, cap, PFMBEM_MIXED, &it, &rs, &rr, true, true, std::sqrt(rn));
      if (si != PFMBEM_OK && si != PFMBEM_ENOCONV) return si;
      iters += it;
      CK(k_axpy(h, cplx{1, 0}, g.c, g.x, (int)n));
    }
    restarts = refinements;
    if (st != PFMBEM_OK && iters < maxit) {
      // refinement stalled above tol (the FP32 operator's accuracy floor, about
      // eps_32 times the condition number, lies above it): finish with FP64
      // GMRES from the current iterate
      int it = 0, rs = 0;
      double rr = relres;
      st = gmres(h, g.b, g.x, tol, maxit - iters, PFMBEM_FP64, &it, &rs, &rr);
      if (st != PFMBEM_OK && st != PFMBEM_ENOCONV) return st;
      iters += it;
      restarts += rs;
      relres = rr;
    }
  } else {
    st = gmres(h, g.b, g.x, tol, maxit, PFMBEM_FP64, &iters, &restarts, &relres, !use_guess);
  }
  // the result and the device error flags come back in one wait
  int* flags = h->hstat;            // [1] tensor-core M2L, [2] device-wide barrier
  if (flags) {
    flags[1] = flags[2] = 0;
    if (h->tc_err) CK(cudaMemcpyAsync(flags + 1, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->fz_err) CK(cudaMemcpyAsync(flags + 2, h->fz_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemcpyAsync(psi, g.x, n * sizeof(cplx), pdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  {
    const pfmbem_status rs = ready_checked(h);
    if (rs != PFMBEM_OK) return rs;
  }
  int tce = 0, fze = 0;
  if (flags) {
    tce = flags[1];
    fze = flags[2];
  } else {
    if (h->tc_err) CK(cudaMemcpy(&tce, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h->fz_err) CK(cudaMemcpy(&fze, h->fz_err, sizeof(int), cudaMemcpyDeviceToHost));
  }
  if (tce) {
    st = PFMBEM_ETIMEOUT;
    h->err = "tensor-core M2L: a bounded wait for the MMA completion gave up";
  }
  if (fze) {
    st = PFMBEM_ETIMEOUT;
    h->err = "single-launch matvec: a bounded device-side wait gave up";
    // the next launch clears the barrier words and this flag first
    h->fz_dirty = true;
  }
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->rel_residual = relres;
    info->ms = now_ms() - t0;
    info->status = st;
  }
  if (st == PFMBEM_ENOCONV) h->err = "GMRES did not reach tol within maxit";
  return st;
}

pfmbem_status pfmbem_lattice_sums(pfmbem_t h, int jmax, double* S) {
  if (!h || !S || jmax < 0 || jmax > 2 * PF_PMAX) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  cplx* Sd = h->stage_out;
  if ((size_t)(jmax + 1) > 2 * (size_t)h->E) return fail(h, PFMBEM_EINVAL, "jmax too large for the work buffer");
  CK(k_lattice_sums(h, jmax, h->lattice_q, Sd));
  std::vector<cplx> tmp(jmax + 1);
  CK(cudaMemcpyAsync(tmp.data(), Sd, sizeof(cplx) * (jmax + 1), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::vector<double> outv(2 * (2 * jmax + 1));
  for (int j = -jmax; j <= jmax; ++j) {
    cplx v = tmp[std::abs(j)];
    outv[2 * (j + jmax)] = v.re;
    outv[2 * (j + jmax) + 1] = v.im;
  }
  if (is_device_ptr(S)) {
    CK(cudaMemcpy(S, outv.data(), sizeof(double) * outv.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(S, outv.data(), sizeof(double) * outv.size());
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_self_terms(pfmbem_t h, double* out) {
  if (!h || !out) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t n = 4 * (size_t)h->E;
  CK(cudaMemcpyAsync(out, h->self4, n * sizeof(cplx), is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PFMBEM_OK;
}

namespace {
// Scattered field and/or its x1-derivative at host or device points (shared by
// pfmbem_field, pfmbem_field_dx1 and pfmbem_etc).
pfmbem_status field_points(pfmbem* h, const double* psi, int npts, const double* pts, double* u, double* du) {
  const size_t n = 2 * (size_t)h->E;
  // host copy of the points for the validity check
  std::vector<double> hp(2 * (size_t)npts);
  if (is_device_ptr(pts)) CK(cudaMemcpy(hp.data(), pts, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost));
  else std::memcpy(hp.data(), pts, sizeof(double) * hp.size());
  // half the block's width: a row of root squares, or the hexagonal cells' extent
  const double ox = h->tree == 1 ? h->wide_cx : h->x0 + 0.5 * h->nroot * h->H;
  const double hw = h->tree == 1 ? h->field_hw : 0.5 * h->nroot * h->H;
  for (int i = 0; i < npts; ++i) {
    if (!std::isfinite(hp[2 * i]) || !std::isfinite(hp[2 * i + 1])) return fail(h, PFMBEM_EINVAL, "non-finite point");
    // the root local expansion of the images |m| >= 2 converges for |x - O| + H/sqrt(2) < 2H
    // (a row of roots or the hexagonal cells: the super root's, of the images
    // |m| >= m0, for |x - C| < 2 R_s)
    if (std::fabs(hp[2 * i] - ox) > hw + 0.2 * h->H)
      return fail(h, PFMBEM_EINVAL, "field point too far from the block along x (|x - centre| > half width + 0.2 H)");
  }
  const cplx* psid;
  pfmbem_status st = stage_input(h, psi, n, h->stage_in, &psid);
  if (st != PFMBEM_OK) return st;
  double2* pd = dalloc_tmp<double2>(h, npts);
  cplx* ud = dalloc_tmp<cplx>(h, 2 * (size_t)npts);
  if (!pd || !ud) return fail(h, PFMBEM_ENOMEM, "field buffers");
  CK(cudaMemcpyAsync(pd, hp.data(), sizeof(double2) * npts, cudaMemcpyHostToDevice, h->stream));
  CK(k_field_prepare(h, psid));
  CK(k_field(h, psid, npts, pd, u ? ud : nullptr, du ? ud + npts : nullptr));
  if (u)
    CK(cudaMemcpyAsync(u, ud, sizeof(cplx) * npts, is_device_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
  if (du)
    CK(cudaMemcpyAsync(du, ud + npts, sizeof(cplx) * npts,
                       is_device_ptr(du) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // release the temporaries
  cudaFreeAsync(pd, h->stream);
  cudaFreeAsync(ud, h->stream);
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)pd), h->allocs.end());
  h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)ud), h->allocs.end());
  return PFMBEM_OK;
}
}  // namespace

pfmbem_status pfmbem_field(pfmbem_t h, const double* psi, int npts, const double* pts, double* u) {
  if (!h || !psi || npts < 0 || (npts > 0 && (!pts || !u))) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  if (npts == 0) return PFMBEM_OK;
  return field_points(h, psi, npts, pts, u, nullptr);
}

pfmbem_status pfmbem_field_dx1(pfmbem_t h, const double* psi, int npts, const double* pts, double* u, double* dudx1) {
  if (!h || !psi || npts < 0 || (npts > 0 && (!pts || (!u && !dudx1)))) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  if (npts == 0) return PFMBEM_OK;
  return field_points(h, psi, npts, pts, u, dudx1);
}

pfmbem_status pfmbem_etc(pfmbem_t h, const double* psi, double x1, int npts, double* etc) {
  if (!h || !psi || !etc || npts < 1 || !std::isfinite(x1)) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  // midpoint rule over one period; |du/dx1| is periodic along x2
  std::vector<double> pts(2 * (size_t)npts);
  for (int i = 0; i < npts; ++i) {
    pts[2 * i] = x1;
    pts[2 * i + 1] = h->y0 + h->H * (i + 0.5) / npts;
  }
  std::vector<cplx> du(npts);
  pfmbem_status st = field_points(h, psi, npts, pts.data(), nullptr, reinterpret_cast<double*>(du.data()));
  if (st != PFMBEM_OK) return st;
  const double c = std::cos(h->theta), s = std::sin(h->theta);
  double sum = 0;
  for (int i = 0; i < npts; ++i) {
    // total field: the incident exp(i k d.x) adds i k cos(theta) exp(i k d.x)
    const double ph = h->k * (c * pts[2 * i] + s * pts[2 * i + 1]);
    const cplx inc{-h->k * c * std::sin(ph), h->k * c * std::cos(ph)};
    sum += std::hypot(du[i].re + inc.re, du[i].im + inc.im);
  }
  *etc = sum * (h->H / npts) / (h->k * h->H);
  return PFMBEM_OK;
}

pfmbem_status pfmbem_coefficients(pfmbem_t h, const double* psi, int max_orders, int* norders, int* orders, double* R,
                                  double* T, double* energy) {
  if (!h || !psi || !norders || max_orders < 0) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const double ks = h->k * std::sin(h->theta);
  std::vector<int> ord;
  int nlo = (int)std::floor((-h->k - ks) * h->H / (2 * M_PI)) - 1;
  int nhi = (int)std::ceil((h->k - ks) * h->H / (2 * M_PI)) + 1;
  for (int n = nlo; n <= nhi; ++n)
    if (std::fabs(ks + 2 * M_PI * n / h->H) < h->k) ord.push_back(n);
  *norders = (int)ord.size();
  if ((int)ord.size() > max_orders || (!ord.empty() && (!orders || !R || !T)))
    return fail(h, PFMBEM_EINVAL, "max_orders smaller than the number of propagating orders");
  const size_t n = 2 * (size_t)h->E;
  const cplx* psid;
  pfmbem_status st = stage_input(h, psi, n, h->stage_in, &psid);
  if (st != PFMBEM_OK) return st;
  const int no = (int)ord.size();
  // order list and results live in the tail of the output staging buffer
  if ((size_t)(2 * no + no) > n) return fail(h, PFMBEM_EINVAL, "too many orders for the work buffer");
  cplx* outd = h->stage_out;
  int* od = reinterpret_cast<int*>(h->stage_out + 2 * no);
  CK(cudaMemcpyAsync(od, ord.data(), sizeof(int) * no, cudaMemcpyHostToDevice, h->stream));
  CK(k_coefficients(h, psid, no, od, outd));
  std::vector<cplx> res(2 * no);
  CK(cudaMemcpyAsync(res.data(), outd, sizeof(cplx) * 2 * no, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double k0 = h->k * std::cos(h->theta);
  double en = 0;
  for (int i = 0; i < no; ++i) {
    cplx t = res[2 * i], r = res[2 * i + 1];
    if (ord[i] == 0) t.re += 1.0;
    orders[i] = ord[i];
    T[2 * i] = t.re;
    T[2 * i + 1] = t.im;
    R[2 * i] = r.re;
    R[2 * i + 1] = r.im;
    const double kap = ks + 2 * M_PI * ord[i] / h->H;
    const double kn = std::sqrt(h->k * h->k - kap * kap);
    en += kn / k0 * (r.re * r.re + r.im * r.im + t.re * t.re + t.im * t.im);
  }
  if (energy) *energy = en;
  return PFMBEM_OK;
}

pfmbem_status pfmbem_warm_features(pfmbem_t h, float* x) {
  if (!h || !x) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t nx = 2 + 3 * (size_t)h->M;
  const bool dev = is_device_ptr(x);
  float* xd = dev ? x : reinterpret_cast<float*>(h->stage_out);
  if (!dev && nx * sizeof(float) > 2 * (size_t)h->E * sizeof(cplx)) return fail(h, PFMBEM_EINVAL, "work buffer");
  CK(k_warm_features(h, xd));
  if (!dev) {
    CK(cudaMemcpyAsync(x, xd, nx * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_warm_features_local(pfmbem_t h, int K, float* x) {
  if (!h || !x || K < 0 || K > 32) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t nx = (size_t)h->M * (5 + 3 * K);
  const bool dev = is_device_ptr(x);
  float* xd = dev ? x : dalloc_tmp<float>(h, nx);
  if (!xd) return fail(h, PFMBEM_ENOMEM, "warm-start buffer");
  CK(k_warm_features_local(h, K, xd));
  if (!dev) {
    CK(cudaMemcpyAsync(x, xd, nx * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    cudaFreeAsync(xd, h->stream);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)xd), h->allocs.end());
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_warm_targets(pfmbem_t h, int nmodes, const double* psi, float* t) {
  if (!h || !psi || !t || nmodes < 0 || nmodes > 64) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t n = 2 * (size_t)h->E, nt = (size_t)h->M * 2 * (2 * nmodes + 1) * 2;
  const cplx* pd;
  pfmbem_status st = stage_input(h, psi, n, h->stage_in, &pd);
  if (st != PFMBEM_OK) return st;
  const bool dev = is_device_ptr(t);
  float* td = dev ? t : dalloc_tmp<float>(h, nt);
  if (!td) return fail(h, PFMBEM_ENOMEM, "warm-start buffer");
  CK(k_warm_targets(h, nmodes, pd, td));
  if (!dev) {
    CK(cudaMemcpyAsync(t, td, nt * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    cudaFreeAsync(td, h->stream);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)td), h->allocs.end());
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_warm_decode(pfmbem_t h, int nmodes, const float* y, double* psi0) {
  if (!h || !y || !psi0 || nmodes < 0 || nmodes > 64) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  const size_t n = 2 * (size_t)h->E, ny = (size_t)h->M * 2 * (2 * nmodes + 1) * 2;
  const bool ydev = is_device_ptr(y);
  float* yd = const_cast<float*>(y);
  if (!ydev) {
    yd = dalloc_tmp<float>(h, ny);
    if (!yd) return fail(h, PFMBEM_ENOMEM, "warm-start buffer");
    CK(cudaMemcpyAsync(yd, y, ny * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  }
  const bool pdev = is_device_ptr(psi0);
  cplx* pd = pdev ? reinterpret_cast<cplx*>(psi0) : h->stage_out;
  CK(k_warm_decode(h, nmodes, yd, pd));
  if (!pdev) CK(cudaMemcpyAsync(psi0, pd, n * sizeof(cplx), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (!ydev) {
    cudaFreeAsync(yd, h->stream);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)yd), h->allocs.end());
  }
  return PFMBEM_OK;
}

pfmbem_status pfmbem_profile(pfmbem_t h, int enable_timing, int reset) {
  if (!h) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  CK(prof_fold(h));
  if (reset) {
    for (int i = 0; i < 32; ++i) {
      h->prof.ms[i] = 0;
      h->prof.launches[i] = 0;
    }
  }
  h->prof.on = enable_timing != 0;
  return PFMBEM_OK;
}

pfmbem_status pfmbem_profile_read(pfmbem_t h, pfmbem_profile_info* out) {
  if (!h || !out) return PFMBEM_EINVAL;
  if (!h->ready) { const pfmbem_status rs = check_ready(h); if (rs != PFMBEM_OK) return rs; }
  CK(cudaStreamSynchronize(h->stream));
  CK(prof_fold(h));
  int64_t tot = 0;
  for (int i = 0; i < 32; ++i) {
    out->ms[i] = h->prof.ms[i];
    out->launches[i] = h->prof.launches[i];
    tot += h->prof.launches[i];
  }
  out->total_launches = tot;
  return PFMBEM_OK;
}

}  // extern "C"
