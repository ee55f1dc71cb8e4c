// Learned warm start for GMRES: a small MLP predicts, from (kH, theta, fiber
// centres and radii), the low Fourier modes of both densities on every fiber;
// decoding them at the element angles gives an initial guess Psi_0.  The
// network is trained on solutions the solver itself produces.  Forward,
// backward and Adam run in the kernels below (FP32).
//
// Layers: in -> hidden (GELU) x layers -> out (linear).  Parameters are one
// flat FP32 array: for every layer W [out][in] row-major, then b [out].
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

struct pfmbem_mlp {
  int in = 0, hidden = 0, layers = 0, out = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> dims;           // layer widths: in, hidden..., out
  std::vector<size_t> woff, boff;  // offsets of W and b of each layer in params
  size_t nparams = 0;
  float* params = nullptr;
  float* grad = nullptr;
  float* m1 = nullptr;             // Adam first moment
  float* m2 = nullptr;             // Adam second moment
  int64_t step = 0;
  int cap = 0;                     // batch capacity of the work buffers
  std::vector<float*> act;         // activations per layer boundary [cap][dims[l]]
  std::vector<float*> pre;         // pre-activations per hidden layer
  float* dA = nullptr;             // work: gradient w.r.t. activations
  float* dB = nullptr;
  float* loss = nullptr;           // device scalar
};

namespace {

constexpr int TS = 16;

// C[M][N] (+)= op(A) op(B) with op given by transA/transB; row-major operands:
//   A is [M][K] (transA = 0) or [K][M] (transA = 1), B is [K][N] or [N][K].
__global__ void gemm_kernel(int M, int N, int K, const float* __restrict__ A, int transA,
                            const float* __restrict__ B, int transB, float* __restrict__ C, int accumulate) {
  __shared__ float As[TS][TS + 1], Bs[TS][TS + 1];
  const int r = blockIdx.y * TS + threadIdx.y, c = blockIdx.x * TS + threadIdx.x;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += TS) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    const int ar = blockIdx.y * TS + threadIdx.y;
    As[threadIdx.y][threadIdx.x] =
        (ar < M && ka < K) ? (transA ? A[(size_t)ka * M + ar] : A[(size_t)ar * K + ka]) : 0.f;
    const int bc = blockIdx.x * TS + threadIdx.x;
    Bs[threadIdx.y][threadIdx.x] =
        (bc < N && kb < K) ? (transB ? B[(size_t)bc * K + kb] : B[(size_t)kb * N + bc]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TS; ++k) acc = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (r < M && c < N) C[(size_t)r * N + c] = accumulate ? C[(size_t)r * N + c] + acc : acc;
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Z[b][o] += bias[o]; then A = gelu(Z) (hidden) or A = Z (output)
__global__ void bias_act_kernel(int B, int O, const float* __restrict__ bias, float* __restrict__ Z,
                                float* __restrict__ Aout, int act) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * O) return;
  const float z = Z[i] + bias[i % O];
  Z[i] = z;
  Aout[i] = act ? gelu(z) : z;
}

// dY = 2 (Y - T) / (B O); loss += sum (Y - T)^2 / (B O)
__global__ void mse_kernel(int n, float scale, const float* __restrict__ Y, const float* __restrict__ T,
                           float* __restrict__ dY, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (i < n) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * d * scale;
    v = d * d * scale;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, v);
}

// db[o] = sum_b dZ[b][o]
__global__ void colsum_kernel(int B, int O, const float* __restrict__ dZ, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(size_t)b * O + o];
  db[o] = s;
}

// dZ = dA * gelu'(Z)
__global__ void gelu_back_kernel(int n, const float* __restrict__ Z, const float* __restrict__ dA,
                                 float* __restrict__ dZ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dA[i] * gelu_grad(Z[i]);
}

__global__ void adam_kernel(size_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                            float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// counter-based uniform in (-1, 1) from (seed, index): SplitMix64
__global__ void init_kernel(size_t n, uint64_t seed, const int64_t* __restrict__ fan_in_of, float* __restrict__ p) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
  const int64_t fi = fan_in_of[i];
  p[i] = fi > 0 ? u * sqrtf(3.f / (float)fi) : 0.f;   // Var = 1/fan_in, biases zero
}

void gemm(cudaStream_t st, int M, int N, int K, const float* A, int ta, const float* B, int tb, float* C, int acc) {
  dim3 blk(TS, TS), grd((N + TS - 1) / TS, (M + TS - 1) / TS);
  gemm_kernel<<<grd, blk, 0, st>>>(M, N, K, A, ta, B, tb, C, acc);
}

cudaError_t ensure_cap(pfmbem_mlp* m, int B) {
  if (B <= m->cap) return cudaSuccess;
  for (float* p : m->act) cudaFree(p);
  for (float* p : m->pre) cudaFree(p);
  cudaFree(m->dA);
  cudaFree(m->dB);
  m->act.assign(m->dims.size(), nullptr);
  m->pre.assign(m->dims.size(), nullptr);
  int wmax = 0;
  for (int d : m->dims) wmax = d > wmax ? d : wmax;
  for (size_t l = 0; l < m->dims.size(); ++l) {
    if (cudaMalloc(&m->act[l], sizeof(float) * (size_t)B * m->dims[l]) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMalloc(&m->pre[l], sizeof(float) * (size_t)B * m->dims[l]) != cudaSuccess) return cudaErrorMemoryAllocation;
  }
  if (cudaMalloc(&m->dA, sizeof(float) * (size_t)B * wmax) != cudaSuccess) return cudaErrorMemoryAllocation;
  if (cudaMalloc(&m->dB, sizeof(float) * (size_t)B * wmax) != cudaSuccess) return cudaErrorMemoryAllocation;
  m->cap = B;
  return cudaSuccess;
}

// forward pass; act[0] must hold the input batch
void forward(pfmbem_mlp* m, int B) {
  const int L = (int)m->dims.size() - 1;
  for (int l = 0; l < L; ++l) {
    const int I = m->dims[l], O = m->dims[l + 1];
    gemm(m->stream, B, O, I, m->act[l], 0, m->params + m->woff[l], 1, m->pre[l + 1], 0);
    bias_act_kernel<<<(B * O + 255) / 256, 256, 0, m->stream>>>(B, O, m->params + m->boff[l], m->pre[l + 1],
                                                                m->act[l + 1], l < L - 1 ? 1 : 0);
  }
}

// backward pass from dY (in m->dA, [B][out]); writes m->grad
void backward(pfmbem_mlp* m, int B) {
  const int L = (int)m->dims.size() - 1;
  float* dcur = m->dA;   // gradient w.r.t. pre-activation of layer l+1
  float* dnext = m->dB;
  for (int l = L - 1; l >= 0; --l) {
    const int I = m->dims[l], O = m->dims[l + 1];
    // dW[o][i] = sum_b dZ[b][o] X[b][i]
    gemm(m->stream, O, I, B, dcur, 1, m->act[l], 0, m->grad + m->woff[l], 0);
    colsum_kernel<<<(O + 127) / 128, 128, 0, m->stream>>>(B, O, dcur, m->grad + m->boff[l]);
    if (l > 0) {
      // dA_prev[b][i] = sum_o dZ[b][o] W[o][i]; then through GELU of layer l
      gemm(m->stream, B, I, O, dcur, 0, m->params + m->woff[l], 0, dnext, 0);
      gelu_back_kernel<<<(B * I + 255) / 256, 256, 0, m->stream>>>(B * I, m->pre[l], dnext, dnext);
      float* t = dcur;
      dcur = dnext;
      dnext = t;
    }
  }
}

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t copy_in(pfmbem_mlp* m, float* dst, const float* src, size_t n) {
  return cudaMemcpyAsync(dst, src, n * sizeof(float), is_dev(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         m->stream);
}

// ---------------------------------------------------------------- features
// x = [kH / 8, theta / (pi/2), then per fiber ((cx - x0)/H, (cy - y0)/H, 4 r / H)]
__global__ void features_kernel(int M, float kH, float th, const double* __restrict__ fc, double x0, double y0,
                                double H, float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    x[0] = kH / 8.f;
    x[1] = th / 1.5707963267948966f;
  }
  if (i < M) {
    x[2 + 3 * i] = (float)((fc[3 * i] - x0) / H);
    x[3 + 3 * i] = (float)((fc[3 * i + 1] - y0) / H);
    x[4 + 3 * i] = (float)(4.0 * fc[3 * i + 2] / H);
  }
}

// Per-fiber network input (one row per fiber, 5 + 3K floats): kH/8,
// theta/(pi/2), 4 r_i/H, the distances (x_i - x_min)/H and (x_max - x_i)/H to
// the block's left and right edges, then the K nearest other fibers in order of
// distance, each as (4 dx/H, 4 dy/H, 4 r_j/H) with dy taken to the nearest
// periodic image; missing neighbours are zeros.  The row depends on positions
// only through differences along y, so a model on these rows is equivariant
// under shifts of the block along the period.  One thread per fiber.
#define PF_WARM_KMAX 32
__global__ void features_local_kernel(int M, int K, float kH, float th, const double* __restrict__ fc, double H,
                                      float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double cx = fc[3 * i], cy = fc[3 * i + 1], ri = fc[3 * i + 2];
  double xmin = 1e300, xmax = -1e300;
  for (int j = 0; j < M; ++j) {
    xmin = fmin(xmin, fc[3 * j] - fc[3 * j + 2]);
    xmax = fmax(xmax, fc[3 * j] + fc[3 * j + 2]);
  }
  double bd[PF_WARM_KMAX];
  int bj[PF_WARM_KMAX];
  double bdy[PF_WARM_KMAX];
  int nb = 0;
  for (int j = 0; j < M; ++j) {
    if (j == i) continue;
    const double dx = fc[3 * j] - cx;
    double dy = fc[3 * j + 1] - cy;
    dy -= H * rint(dy / H);
    const double d2 = dx * dx + dy * dy;
    // insertion into the K nearest so far
    int pos = nb < K ? nb : K;
    while (pos > 0 && bd[pos - 1] > d2) {
      if (pos < K) { bd[pos] = bd[pos - 1]; bj[pos] = bj[pos - 1]; bdy[pos] = bdy[pos - 1]; }
      --pos;
    }
    if (pos < K) {
      bd[pos] = d2;
      bj[pos] = j;
      bdy[pos] = dy;
      if (nb < K) ++nb;
    }
  }
  float* o = x + (size_t)i * (5 + 3 * K);
  o[0] = kH / 8.f;
  o[1] = th / 1.5707963267948966f;
  o[2] = (float)(4.0 * ri / H);
  o[3] = (float)((cx - xmin) / H);
  o[4] = (float)((xmax - cx) / H);
  for (int q = 0; q < K; ++q) {
    float* v = o + 5 + 3 * q;
    if (q < nb) {
      const int j = bj[q];
      v[0] = (float)(4.0 * (fc[3 * j] - cx) / H);
      v[1] = (float)(4.0 * bdy[q] / H);
      v[2] = (float)(4.0 * fc[3 * j + 2] / H);
    } else {
      v[0] = v[1] = v[2] = 0.f;
    }
  }
}

// Fourier coefficients of a solution: for fiber i, density d, mode n = -8..8,
//   c = (1/N_i) sum_e psi_{e,d} e^{-i n t_e} e^{-i k c_i.dir},
// t_e = angle of c_e about c_i measured from the incidence direction, so that an
// isolated circle's response has the same coefficients at every incidence angle.
// One block per (fiber, density); threads over modes.
__global__ void targets_kernel(int M, int nm, const int* __restrict__ foff, const double* __restrict__ fc,
                               const double2* __restrict__ oc, double k, double dx, double dy,
                               const cplx* __restrict__ psi, float* __restrict__ t) {
  const int i = blockIdx.x >> 1, d = blockIdx.x & 1;
  const int n = (int)threadIdx.x - nm;
  if (threadIdx.x >= 2 * nm + 1) return;
  const int f0 = foff[i], N = foff[i + 1] - f0;
  const double cx = fc[3 * i], cy = fc[3 * i + 1];
  cplx acc{0, 0};
  for (int e = f0; e < f0 + N; ++e) {
    // angle of (c_e - c_i) relative to dir = (dx, dy)
    const double ux = oc[e].x - cx, uy = oc[e].y - cy;
    const double te = atan2(uy * dx - ux * dy, ux * dx + uy * dy);
    double s, c;
    sincos(-n * te, &s, &c);
    acc += psi[2 * e + d] * cplx{c, s};
  }
  double s, c;
  sincos(-k * (cx * dx + cy * dy), &s, &c);
  acc = (1.0 / N) * (acc * cplx{c, s});
  const size_t o = (((size_t)i * 2 + d) * (2 * nm + 1) + (n + nm)) * 2;
  t[o] = (float)acc.re;
  t[o + 1] = (float)acc.im;
}

// psi0_{e,d} = e^{i k c_i.dir} sum_n c_{i,d,n} e^{i n t_e} (t_e as above); one thread per element.
__global__ void decode_kernel(int E, int nm, const int* __restrict__ fib, const double* __restrict__ fc,
                              const double2* __restrict__ oc, double k, double dx, double dy,
                              const float* __restrict__ y, cplx* __restrict__ psi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = fib[e];
  const double cx = fc[3 * i], cy = fc[3 * i + 1];
  const double ux = oc[e].x - cx, uy = oc[e].y - cy;
  const double te = atan2(uy * dx - ux * dy, ux * dx + uy * dy);
  double s, c;
  sincos(k * (cx * dx + cy * dy), &s, &c);
  const cplx ph{c, s};
  for (int d = 0; d < 2; ++d) {
    cplx acc{0, 0};
    for (int n = -nm; n <= nm; ++n) {
      const size_t o = (((size_t)i * 2 + d) * (2 * nm + 1) + (n + nm)) * 2;
      double sn, cn;
      sincos(n * te, &sn, &cn);
      acc += cplx{(double)y[o], (double)y[o + 1]} * cplx{cn, sn};
    }
    psi[2 * e + d] = ph * acc;
  }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

pfmbem_status pfmbem_mlp_create(int in, int hidden, int layers, int out, uint64_t seed, void* stream,
                                pfmbem_mlp_t* res) {
  if (!res || in < 1 || hidden < 1 || layers < 1 || out < 1 || layers > 16) return PFMBEM_EINVAL;
  *res = nullptr;
  pfmbem_mlp* m = new pfmbem_mlp();
  m->in = in;
  m->hidden = hidden;
  m->layers = layers;
  m->out = out;
  m->stream = static_cast<cudaStream_t>(stream);
  m->dims.push_back(in);
  for (int l = 0; l < layers; ++l) m->dims.push_back(hidden);
  m->dims.push_back(out);
  size_t off = 0;
  std::vector<int64_t> fan;
  for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
    const size_t nw = (size_t)m->dims[l] * m->dims[l + 1];
    m->woff.push_back(off);
    off += nw;
    m->boff.push_back(off);
    off += m->dims[l + 1];
    fan.insert(fan.end(), nw, m->dims[l]);
    fan.insert(fan.end(), m->dims[l + 1], 0);
  }
  m->nparams = off;
  int64_t* fan_d = nullptr;
  if (cudaMalloc(&m->params, off * sizeof(float)) != cudaSuccess || cudaMalloc(&m->grad, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&m->m1, off * sizeof(float)) != cudaSuccess || cudaMalloc(&m->m2, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&fan_d, off * sizeof(int64_t)) != cudaSuccess) {
    pfmbem_mlp_destroy(m);
    return PFMBEM_ENOMEM;
  }
  cudaMemcpyAsync(fan_d, fan.data(), off * sizeof(int64_t), cudaMemcpyHostToDevice, m->stream);
  init_kernel<<<(unsigned)((off + 255) / 256), 256, 0, m->stream>>>(off, seed, fan_d, m->params);
  cudaMemsetAsync(m->m1, 0, off * sizeof(float), m->stream);
  cudaMemsetAsync(m->m2, 0, off * sizeof(float), m->stream);
  cudaStreamSynchronize(m->stream);
  cudaFree(fan_d);
  if (cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
    pfmbem_mlp_destroy(m);
    return PFMBEM_ENOMEM;
  }
  if (cudaGetLastError() != cudaSuccess) {
    pfmbem_mlp_destroy(m);
    return PFMBEM_ECUDA;
  }
  *res = m;
  return PFMBEM_OK;
}

void pfmbem_mlp_destroy(pfmbem_mlp_t m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->params);
  cudaFree(m->grad);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->loss);
  for (float* p : m->act) cudaFree(p);
  for (float* p : m->pre) cudaFree(p);
  cudaFree(m->dA);
  cudaFree(m->dB);
  delete m;
}

pfmbem_status pfmbem_mlp_params(pfmbem_mlp_t m, int64_t* nparams, float* get, const float* set) {
  if (!m || !nparams) return PFMBEM_EINVAL;
  *nparams = (int64_t)m->nparams;
  if (set && copy_in(m, m->params, set, m->nparams) != cudaSuccess) return PFMBEM_ECUDA;
  if (get) {
    if (cudaMemcpyAsync(get, m->params, m->nparams * sizeof(float),
                        is_dev(get) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
      return PFMBEM_ECUDA;
  }
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PFMBEM_OK : PFMBEM_ECUDA;
}

pfmbem_status pfmbem_mlp_forward(pfmbem_mlp_t m, int B, const float* X, float* Y) {
  if (!m || B < 1 || !X || !Y) return PFMBEM_EINVAL;
  if (ensure_cap(m, B) != cudaSuccess) return PFMBEM_ENOMEM;
  if (copy_in(m, m->act[0], X, (size_t)B * m->in) != cudaSuccess) return PFMBEM_ECUDA;
  forward(m, B);
  if (cudaMemcpyAsync(Y, m->act.back(), sizeof(float) * (size_t)B * m->out,
                      is_dev(Y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PFMBEM_ECUDA;
  if (!is_dev(Y) && cudaStreamSynchronize(m->stream) != cudaSuccess) return PFMBEM_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PFMBEM_OK : PFMBEM_ECUDA;
}

// Mean-squared error over the batch and, if grad != NULL, its gradient with
// respect to every parameter (flat layout); lr > 0 additionally takes one Adam
// step (beta1 0.9, beta2 0.999, eps 1e-8).
pfmbem_status pfmbem_mlp_train(pfmbem_mlp_t m, int B, const float* X, const float* T, float lr, float* loss,
                               float* grad) {
  if (!m || B < 1 || !X || !T) return PFMBEM_EINVAL;
  if (ensure_cap(m, B) != cudaSuccess) return PFMBEM_ENOMEM;
  if (copy_in(m, m->act[0], X, (size_t)B * m->in) != cudaSuccess) return PFMBEM_ECUDA;
  if (copy_in(m, m->dB, T, (size_t)B * m->out) != cudaSuccess) return PFMBEM_ECUDA;
  forward(m, B);
  cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
  const int n = B * m->out;
  // the target is parked in dB; dY goes to dA
  mse_kernel<<<(n + 255) / 256, 256, 0, m->stream>>>(n, 1.f / (float)n, m->act.back(), m->dB, m->dA, m->loss);
  backward(m, B);
  if (lr > 0) {
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - (float)std::pow(b1, (double)m->step));
    const float c2 = 1.f / (1.f - (float)std::pow(b2, (double)m->step));
    adam_kernel<<<(unsigned)((m->nparams + 255) / 256), 256, 0, m->stream>>>(m->nparams, lr, b1, b2, 1e-8f, c1, c2,
                                                                            m->params, m->grad, m->m1, m->m2);
  }
  if (grad && cudaMemcpyAsync(grad, m->grad, m->nparams * sizeof(float),
                              is_dev(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PFMBEM_ECUDA;
  if (loss && cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PFMBEM_ECUDA;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return PFMBEM_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PFMBEM_OK : PFMBEM_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- handle side
cudaError_t k_warm_features(pfmbem* h, float* x_dev) {
  features_kernel<<<(h->M + 127) / 128, 128, 0, h->stream>>>(h->M, (float)(h->k * h->H), (float)h->theta, h->fib_geo,
                                                             h->x0, h->y0, h->H, x_dev);
  return cudaGetLastError();
}

cudaError_t k_warm_features_local(pfmbem* h, int K, float* x_dev) {
  features_local_kernel<<<(h->M + 127) / 128, 128, 0, h->stream>>>(h->M, K, (float)(h->k * h->H), (float)h->theta,
                                                                   h->fib_geo, h->H, x_dev);
  return cudaGetLastError();
}

cudaError_t k_warm_targets(pfmbem* h, int nm, const cplx* psi, float* t_dev) {
  targets_kernel<<<2 * h->M, 32 * ((2 * nm + 1 + 31) / 32), 0, h->stream>>>(h->M, nm, h->fib_off, h->fib_geo, h->o_c, h->k,
                                                                              cos(h->theta), sin(h->theta), psi, t_dev);
  return cudaGetLastError();
}

cudaError_t k_warm_decode(pfmbem* h, int nm, const float* y_dev, cplx* psi) {
  decode_kernel<<<(h->E + 127) / 128, 128, 0, h->stream>>>(h->E, nm, h->o_fiber, h->fib_geo, h->o_c, h->k,
                                                          cos(h->theta), sin(h->theta), y_dev, psi);
  return cudaGetLastError();
}
