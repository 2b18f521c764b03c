// Learned warm start of the eigenvalue solve (not part of the paper: its
// Algorithm 1 starts at 1/E).  A small MLP maps 64 log-spectrum quantiles per
// axis (+ 4 scale features) to 64 quantiles of log(lam E) per axis.  Forward,
// backward (MSE) and Adam run in these SIMT kernels; the plain solve always
// runs to its tolerance from the predicted start, so the network can only
// change the iteration count, never the answer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {
namespace {

constexpr int kNQ = 64;
constexpr int kIn = GMGM_MLP_IN, kH = GMGM_MLP_HIDDEN, kOut = GMGM_MLP_OUT;

// offsets of the flat parameter vector: W1 [kH][kIn], b1, W2 [kH][kH], b2, W3 [kOut][kH], b3
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, oEnd = ob3 + kOut;
static_assert(oEnd == GMGM_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ double interp_at(const double* v, int r, double pos) {
  int lo = int(floor(pos));
  lo = lo < 0 ? 0 : (lo > r - 1 ? r - 1 : lo);
  const int hi = lo + 1 < r ? lo + 1 : r - 1;
  const double fr = pos - lo;
  return v[lo] * (1.0 - fr) + v[hi] * fr;
}

// log E quantiles (minus log mean) per axis + 4 extras; one block.
__global__ void features_kernel(const double* __restrict__ E0, int r0, const double* __restrict__ E1, int r1,
                                float* __restrict__ out) {
  __shared__ double red[33];
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < r0; i += blockDim.x) s0 += E0[i];
  for (int i = threadIdx.x; i < r1; i += blockDim.x) s1 += E1[i];
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  for (int k = threadIdx.x; k < 2 * kNQ; k += blockDim.x) {
    const int a = k / kNQ, q = k % kNQ;
    const double* E = a ? E1 : E0;
    const int r = a ? r1 : r0;
    const double pos = double(q) / (kNQ - 1) * (r - 1);
    int lo = int(floor(pos));
    const int hi = lo + 1 < r ? lo + 1 : r - 1;
    const double fr = pos - lo;
    const double v = log(E[lo]) * (1.0 - fr) + log(E[hi]) * fr;
    out[k] = float(v - log((a ? s1 : s0) / r));
  }
  if (threadIdx.x == 0) {
    out[2 * kNQ + 0] = float(log(double(r0)) / 8.0);
    out[2 * kNQ + 1] = float(log(double(r1)) / 8.0);
    out[2 * kNQ + 2] = float(log(s0) - log(s1));
    out[2 * kNQ + 3] = float(log(E0[0]) - log(E1[0]));
  }
}

__global__ void targets_kernel(const double* __restrict__ E0, int r0, const double* __restrict__ E1, int r1,
                               const double* __restrict__ l0, const double* __restrict__ l1, float* __restrict__ out) {
  for (int k = threadIdx.x; k < 2 * kNQ; k += blockDim.x) {
    const int a = k / kNQ, q = k % kNQ;
    const double* E = a ? E1 : E0;
    const double* L = a ? l1 : l0;
    const int r = a ? r1 : r0;
    const double pos = double(q) / (kNQ - 1) * (r - 1);
    int lo = int(floor(pos));
    const int hi = lo + 1 < r ? lo + 1 : r - 1;
    const double fr = pos - lo;
    out[k] = float(log(L[lo] * E[lo]) * (1.0 - fr) + log(L[hi] * E[hi]) * fr);
  }
}

// lam_i = exp(interp of y at i/(r-1)*63) / E_i, clipped at eps; falls back
// to Algorithm 1's 1/E for the whole axis if anything is not finite.
__global__ void expand_kernel(const float* __restrict__ y, const double* __restrict__ E0, int r0,
                              const double* __restrict__ E1, int r1, double eps, double* __restrict__ l0,
                              double* __restrict__ l1) {
  __shared__ int bad[2];
  __shared__ double yq[2 * kNQ];
  if (threadIdx.x < 2) bad[threadIdx.x] = 0;
  for (int k = threadIdx.x; k < 2 * kNQ; k += blockDim.x) yq[k] = double(y[k]);
  __syncthreads();
  for (int a = 0; a < 2; ++a) {
    const double* E = a ? E1 : E0;
    double* L = a ? l1 : l0;
    const int r = a ? r1 : r0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      const double pos = r > 1 ? double(i) / (r - 1) * (kNQ - 1) : 0.0;
      const double v = exp(interp_at(yq + a * kNQ, kNQ, pos)) / E[i];
      if (!isfinite(v) || !(v > 0.0)) atomicOr(&bad[a], 1);
      L[i] = fmax(v, eps);
    }
  }
  __syncthreads();
  for (int a = 0; a < 2; ++a) {
    if (!bad[a]) continue;
    const double* E = a ? E1 : E0;
    double* L = a ? l1 : l0;
    const int r = a ? r1 : r0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) L[i] = fmax(1.0 / E[i], eps);
  }
}

// Y[b][o] = act(sum_i X[b][i] W[o][i] + bias[o])
__global__ void linear_fwd_kernel(const float* __restrict__ X, int B, int nin, const float* __restrict__ W,
                                  const float* __restrict__ bias, int nout, int relu, float* __restrict__ Y) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (o >= nout || b >= B) return;
  const float* x = X + int64_t(b) * nin;
  const float* w = W + int64_t(o) * nin;
  float s = bias[o];
  for (int i = 0; i < nin; ++i) s = fmaf(x[i], w[i], s);
  Y[int64_t(b) * nout + o] = relu ? fmaxf(s, 0.f) : s;
}

// dY = 2 (Y - T) / (B nout); loss partial sums into *loss (atomic)
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, int64_t n, float* __restrict__ dY,
                                float* __restrict__ loss) {
  float acc = 0.f;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = 2.f * d / float(n);
    acc += d * d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / float(n));
}

// dZ = dA * (A > 0) in place (A is the post-ReLU activation)
__global__ void relu_bwd_kernel(const float* __restrict__ A, float* __restrict__ dA, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    if (!(A[e] > 0.f)) dA[e] = 0.f;
}

// gW[o][i] = sum_b dZ[b][o] X[b][i]; gb[o] = sum_b dZ[b][o]
__global__ void linear_wgrad_kernel(const float* __restrict__ dZ, const float* __restrict__ X, int B, int nin, int nout,
                                    float* __restrict__ gW, float* __restrict__ gb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;
  if (o >= nout) return;
  if (i < nin) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s = fmaf(dZ[int64_t(b) * nout + o], X[int64_t(b) * nin + i], s);
    gW[int64_t(o) * nin + i] = s;
  }
  if (i == 0) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[int64_t(b) * nout + o];
    gb[o] = s;
  }
}

// dX[b][i] = sum_o dZ[b][o] W[o][i]
__global__ void linear_xgrad_kernel(const float* __restrict__ dZ, const float* __restrict__ W, int B, int nin, int nout,
                                    float* __restrict__ dX) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= nin || b >= B) return;
  float s = 0.f;
  for (int o = 0; o < nout; ++o) s = fmaf(dZ[int64_t(b) * nout + o], W[int64_t(o) * nin + i], s);
  dX[int64_t(b) * nin + i] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, int width, const int* __restrict__ idx, int B,
                                   float* __restrict__ dst) {
  const int64_t n = int64_t(B) * width;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = e / width, c = e - b * width;
    dst[e] = src[int64_t(idx[b]) * width + c];
  }
}

struct Acts {
  float *a1, *a2, *y, *d2, *d1, *dy;
};

void forward(cudaStream_t s, const float* P, const float* X, int B, Acts A) {
  linear_fwd_kernel<<<dim3((kH + 127) / 128, B), 128, 0, s>>>(X, B, kIn, P + oW1, P + ob1, kH, 1, A.a1);
  linear_fwd_kernel<<<dim3((kH + 127) / 128, B), 128, 0, s>>>(A.a1, B, kH, P + oW2, P + ob2, kH, 1, A.a2);
  linear_fwd_kernel<<<dim3((kOut + 127) / 128, B), 128, 0, s>>>(A.a2, B, kH, P + oW3, P + ob3, kOut, 0, A.y);
}

// loss (device scalar, accumulated) and gradient G (flat) of the MSE
void backward(cudaStream_t s, const float* P, const float* X, const float* T, int B, Acts A, float* G, float* loss) {
  const int64_t ny = int64_t(B) * kOut, nh = int64_t(B) * kH;
  mse_grad_kernel<<<64, 256, 0, s>>>(A.y, T, ny, A.dy, loss);
  linear_wgrad_kernel<<<dim3((kH + 127) / 128, kOut), 128, 0, s>>>(A.dy, A.a2, B, kH, kOut, G + oW3, G + ob3);
  linear_xgrad_kernel<<<dim3((kH + 127) / 128, B), 128, 0, s>>>(A.dy, P + oW3, B, kH, kOut, A.d2);
  relu_bwd_kernel<<<64, 256, 0, s>>>(A.a2, A.d2, nh);
  linear_wgrad_kernel<<<dim3((kH + 127) / 128, kH), 128, 0, s>>>(A.d2, A.a1, B, kH, kH, G + oW2, G + ob2);
  linear_xgrad_kernel<<<dim3((kH + 127) / 128, B), 128, 0, s>>>(A.d2, P + oW2, B, kH, kH, A.d1);
  relu_bwd_kernel<<<64, 256, 0, s>>>(A.a1, A.d1, nh);
  linear_wgrad_kernel<<<dim3((kIn + 127) / 128, kH), 128, 0, s>>>(A.d1, X, B, kIn, kH, G + oW1, G + ob1);
}

Acts carve_acts(Carve& c, int B) {
  Acts A;
  A.a1 = c.take<float>(size_t(B) * kH);
  A.a2 = c.take<float>(size_t(B) * kH);
  A.y = c.take<float>(size_t(B) * kOut);
  A.d2 = c.take<float>(size_t(B) * kH);
  A.d1 = c.take<float>(size_t(B) * kH);
  A.dy = c.take<float>(size_t(B) * kOut);
  return A;
}

size_t acts_bytes(int B) { return (size_t(B) * (4 * kH + 2 * kOut)) * 4 + 8 * 256; }

}  // namespace

size_t mlp_scratch_bytes(int batch, int64_t steps) {
  return acts_bytes(batch) + Carve::round(size_t(GMGM_MLP_PARAMS) * 4) + Carve::round(size_t(batch) * (kIn + kOut) * 4) +
         Carve::round(size_t(std::max<int64_t>(steps, 1)) * batch * 4) + 4096;
}

cudaError_t launch_features(gmgm_handle* h, const double* E0, int r0, const double* E1, int r1, float* out) {
  features_kernel<<<1, 128, 0, h->stream>>>(E0, r0, E1, r1, out);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_targets(gmgm_handle* h, const double* E0, int r0, const double* E1, int r1, const double* l0,
                           const double* l1, float* out) {
  targets_kernel<<<1, 128, 0, h->stream>>>(E0, r0, E1, r1, l0, l1, out);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t mlp_forward(gmgm_handle* h, const float* P, const float* X, int B, float* out, void* scratch) {
  Carve c(scratch);
  Acts A = carve_acts(c, B);
  forward(h->stream, P, X, B, A);
  note_launch(3);
  return cudaMemcpyAsync(out, A.y, size_t(B) * kOut * 4, cudaMemcpyDeviceToDevice, h->stream);
}

cudaError_t mlp_loss_grad(gmgm_handle* h, const float* P, const float* X, const float* T, int B, float* G,
                          float* loss_dev, void* scratch) {
  Carve c(scratch);
  Acts A = carve_acts(c, B);
  float* Gs = G ? G : c.take<float>(GMGM_MLP_PARAMS);
  cudaError_t e = cudaMemsetAsync(loss_dev, 0, 4, h->stream);
  if (e != cudaSuccess) return e;
  forward(h->stream, P, X, B, A);
  backward(h->stream, P, X, T, B, A, Gs, loss_dev);
  note_launch(11);
  return cudaGetLastError();
}

cudaError_t mlp_train(gmgm_handle* h, float* P, float* adam, const float* X, const float* T, int n,
                      const gmgm_train_opts* o, float* loss_dev, void* scratch) {
  const int B = std::min(o->batch, n);
  Carve c(scratch);
  Acts A = carve_acts(c, B);
  float* G = c.take<float>(GMGM_MLP_PARAMS);
  float* Xb = c.take<float>(size_t(B) * kIn);
  float* Tb = c.take<float>(size_t(B) * kOut);
  int* idx = c.take<int>(size_t(std::max(o->steps, 1)) * B);
  // mini-batch order: a seeded shuffle per epoch, drawn on the host
  std::vector<int> hidx(size_t(std::max(o->steps, 1)) * B);
  std::mt19937_64 rng(o->seed);
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  size_t pos = size_t(n);
  for (size_t t = 0; t < hidx.size(); ++t) {
    if (pos >= size_t(n)) {
      std::shuffle(perm.begin(), perm.end(), rng);
      pos = 0;
    }
    hidx[t] = perm[pos++];
  }
  cudaError_t e = cudaMemcpyAsync(idx, hidx.data(), hidx.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return e;  // hidx outlives the copy
  float* m = adam;
  float* v = adam + GMGM_MLP_PARAMS;
  float c1 = 1.f, c2 = 1.f;
  for (int step = 0; step < o->steps; ++step) {
    gather_rows_kernel<<<64, 256, 0, h->stream>>>(X, kIn, idx + size_t(step) * B, B, Xb);
    gather_rows_kernel<<<64, 256, 0, h->stream>>>(T, kOut, idx + size_t(step) * B, B, Tb);
    if ((e = cudaMemsetAsync(loss_dev, 0, 4, h->stream)) != cudaSuccess) return e;
    forward(h->stream, P, Xb, B, A);
    backward(h->stream, P, Xb, Tb, B, A, G, loss_dev);
    c1 *= o->beta1;
    c2 *= o->beta2;
    adam_kernel<<<128, 256, 0, h->stream>>>(P, G, m, v, GMGM_MLP_PARAMS, o->lr, o->beta1, o->beta2, o->eps, 1.f - c1,
                                            1.f - c2);
    note_launch(14);
  }
  return cudaGetLastError();
}

cudaError_t warmstart_infer(gmgm_handle* h, const float* P, const double* E0, int r0, const double* E1, int r1,
                            double eps, double* l0, double* l1, void* scratch) {
  Carve c(scratch);
  Acts A = carve_acts(c, 1);
  float* f = c.take<float>(kIn);
  features_kernel<<<1, 128, 0, h->stream>>>(E0, r0, E1, r1, f);
  forward(h->stream, P, f, 1, A);
  expand_kernel<<<1, 256, 0, h->stream>>>(A.y, E0, r0, E1, r1, eps, l0, l1);
  note_launch(5);
  return cudaGetLastError();
}

}  // namespace gmgm
