// The learned correction network of the PHSVDS solver (the learned-
// preconditioner form; the paper's own preconditioners are Sec. 4): a 3-layer
// 3x3 convolution network 4 -> 16 -> 16 -> 1 channels with ReLU and no
// biases, BF16 weights and FP32 arithmetic, on the operator's grid.
//
// Images are planar: x[b][c][y][x], one plane of nx*ny floats per channel.
// Parameters (3024 BF16 values) are layer-major, each layer [o][c][p][q].
//
// A 3x3 convolution with 16 channels is a contraction of length 9*16 = 144 per
// output pixel; at the grid sizes of the solver (<= 65,536 pixels) it is a few
// MFLOP per image, so it runs on the FP32 pipes from shared-memory tiles (one
// 16x16 output tile per CTA, the input tile with its one-pixel halo and the
// layer's weights staged once) rather than on the tensor cores.
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "kernels.h"
#include "phsvds.h"

namespace ph {

constexpr int CNN_T = 16;            // output tile side
constexpr int CNN_H = CNN_T + 2;     // tile with halo
constexpr int CNN_NPARAM = 16 * 4 * 9 + 16 * 16 * 9 + 1 * 16 * 9;

// out[b][o] = conv(in[b], w) (3x3, zero padding); then ReLU if relu; then
// zeroed where mask[b][o] <= 0 if mask != nullptr (the ReLU derivative of the
// layer whose output the mask is).  w: float [O][C][9].
template <int C, int O>
__global__ void __launch_bounds__(256) k_conv3(int nx, int ny, const float* __restrict__ in,
                                               const float* __restrict__ w, float* __restrict__ out, int relu,
                                               const float* __restrict__ mask) {
  __shared__ float tile[C][CNN_H][CNN_H + 1];
  __shared__ float ws[O * C * 9];
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * CNN_T, y0 = blockIdx.y * CNN_T;
  const int tid = threadIdx.x;
  const size_t plane = (size_t)nx * ny;
  for (int i = tid; i < O * C * 9; i += 256) ws[i] = w[i];
  const float* inb = in + (size_t)b * C * plane;
  for (int i = tid; i < C * CNN_H * CNN_H; i += 256) {
    const int c = i / (CNN_H * CNN_H), r = i % (CNN_H * CNN_H);
    const int ty = r / CNN_H, tx = r % CNN_H;
    const int gy = y0 + ty - 1, gx = x0 + tx - 1;
    tile[c][ty][tx] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? inb[c * plane + (size_t)gy * nx + gx] : 0.f;
  }
  __syncthreads();
  const int ly = tid / CNN_T, lx = tid % CNN_T;
  float acc[O];
#pragma unroll
  for (int o = 0; o < O; ++o) acc[o] = 0.f;
  for (int c = 0; c < C; ++c) {
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const float v = tile[c][ly + t / 3][lx + t % 3];
#pragma unroll
      for (int o = 0; o < O; ++o) acc[o] = fmaf(ws[(o * C + c) * 9 + t], v, acc[o]);
    }
  }
  const int gy = y0 + ly, gx = x0 + lx;
  if (gy < ny && gx < nx) {
    const size_t pix = (size_t)gy * nx + gx;
#pragma unroll
    for (int o = 0; o < O; ++o) {
      float r = relu ? fmaxf(acc[o], 0.f) : acc[o];
      if (mask && !(mask[((size_t)b * O + o) * plane + pix] > 0.f)) r = 0.f;
      out[((size_t)b * O + o) * plane + pix] = r;
    }
  }
}

// dw[o][c][t] += sum_b sum_pix g[b][o][pix] * a[b][c][pix + tap t]: the weight
// gradient of out = conv(a, w), reduced over one tile per CTA, then added to
// dw with one atomic per weight.
template <int C, int O>
__global__ void __launch_bounds__(256) k_conv3_wgrad(int nx, int ny, const float* __restrict__ a,
                                                     const float* __restrict__ g, float* __restrict__ dw) {
  __shared__ float at[C][CNN_H][CNN_H + 1];
  __shared__ float gt[O][CNN_T][CNN_T + 1];
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * CNN_T, y0 = blockIdx.y * CNN_T;
  const int tid = threadIdx.x;
  const size_t plane = (size_t)nx * ny;
  const float* ab = a + (size_t)b * C * plane;
  const float* gb = g + (size_t)b * O * plane;
  for (int i = tid; i < C * CNN_H * CNN_H; i += 256) {
    const int c = i / (CNN_H * CNN_H), r = i % (CNN_H * CNN_H);
    const int ty = r / CNN_H, tx = r % CNN_H;
    const int gy = y0 + ty - 1, gx = x0 + tx - 1;
    at[c][ty][tx] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? ab[c * plane + (size_t)gy * nx + gx] : 0.f;
  }
  for (int i = tid; i < O * CNN_T * CNN_T; i += 256) {
    const int o = i / (CNN_T * CNN_T), r = i % (CNN_T * CNN_T);
    const int ty = r / CNN_T, tx = r % CNN_T;
    const int gy = y0 + ty, gx = x0 + tx;
    gt[o][ty][tx] = (gy < ny && gx < nx) ? gb[o * plane + (size_t)gy * nx + gx] : 0.f;
  }
  __syncthreads();
  for (int i = tid; i < O * C * 9; i += 256) {
    const int o = i / (C * 9), r = i % (C * 9), c = r / 9, t = r % 9, p = t / 3, q = t % 3;
    float s = 0.f;
    for (int ly = 0; ly < CNN_T; ++ly)
#pragma unroll 4
      for (int lx = 0; lx < CNN_T; ++lx) s = fmaf(gt[o][ly][lx], at[c][ly + p][lx + q], s);
    atomicAdd(dw + i, s);
  }
}

// Forward and transposed-flipped FP32 weights from the BF16 parameters:
// wf = params as float; wt (layers 2 and 3) [c][o][8 - t] = w[o][c][t], the
// weights of the input-gradient convolution.
__global__ void k_cnn_weights(const __nv_bfloat16* __restrict__ p, float* __restrict__ wf, float* __restrict__ wt) {
  const int L1 = 16 * 4 * 9, L2 = 16 * 16 * 9, L3 = 16 * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CNN_NPARAM; i += gridDim.x * blockDim.x) {
    const float v = __bfloat162float(p[i]);
    wf[i] = v;
    if (i < L1) continue;
    if (i < L1 + L2) {
      const int k = i - L1, o = k / (16 * 9), c = (k / 9) % 16, t = k % 9;
      wt[L1 + (c * 16 + o) * 9 + (8 - t)] = v;
    } else {
      const int k = i - L1 - L2, c = k / 9, t = k % 9;   // o = 0
      (void)L3;
      wt[L1 + L2 + c * 9 + (8 - t)] = v;
    }
  }
}

// Per-sample loss and gradient of L = (1/B) sum_b ||y_b - t_b||^2 / ||t_b||^2:
// tn2[b] = ||t_b||^2 must be computed first (k_sample_norm2).
__global__ void k_sample_norm2(int npix, const float* __restrict__ t, double* __restrict__ tn2) {
  const int b = blockIdx.y;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    const double v = t[(size_t)b * npix + i];
    s += v * v;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(tn2 + b, s);
}

__global__ void k_cnn_loss(int B, int npix, const float* __restrict__ y, const float* __restrict__ t,
                           const double* __restrict__ tn2, float* __restrict__ g, double* __restrict__ loss) {
  const int b = blockIdx.y;
  const double inv = 1.0 / (B * fmax(tn2[b], 1e-300));
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    const size_t k = (size_t)b * npix + i;
    const double d = (double)y[k] - (double)t[k];
    g[k] = (float)(2.0 * d * inv);
    s += d * d * inv;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// Adam on the FP32 master weights, then round to the BF16 parameters; zeroes
// the gradient for the next accumulation.
__global__ void k_cnn_adam(int n, float* __restrict__ w, float* __restrict__ gr, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                           __nv_bfloat16* __restrict__ p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    p[i] = __float2bfloat16_rn(wi);
    gr[i] = 0.f;
  }
}

// Solver side: image b of x = [r_b * scale_b, f0, f1, f2] for the columns of
// the residual block R (n x nb, column-major, ld ldr), scale_b = sqrt(n) /
// ||r_b|| from norms2[b] = ||r_b||^2 (a zero column gives a zero image).
template <typename T>
__global__ void k_cnn_pack(int n, int nb, const T* __restrict__ R, int ldr, const double* __restrict__ norms2,
                           const float* __restrict__ feat, float* __restrict__ x) {
  const int b = blockIdx.y;
  const double nr = norms2[b];
  const float sc = nr > 0.0 ? (float)sqrt((double)n / nr) : 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float* xb = x + (size_t)b * 4 * n;
    xb[i] = (float)R[(size_t)b * ldr + i] * sc;
    xb[n + i] = feat[i];
    xb[2 * n + i] = feat[n + i];
    xb[3 * n + i] = feat[2 * n + i];
  }
}

// t_b = y_b (the network output; its scale is irrelevant to the subspace
// method) into the column-major correction block.
template <typename T>
__global__ void k_cnn_unpack(int n, int nb, const float* __restrict__ y, T* __restrict__ Tb, int ldt) {
  const int b = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Tb[(size_t)b * ldt + i] = (T)y[(size_t)b * n + i];
}

// ---------------------------------------------------------------------------
static dim3 tiles(int nx, int ny, int B) { return dim3((nx + CNN_T - 1) / CNN_T, (ny + CNN_T - 1) / CNN_T, B); }

void cnn_weights(cudaStream_t s, const void* params_bf16, float* wf, float* wt) {
  k_cnn_weights<<<(CNN_NPARAM + 255) / 256, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(params_bf16), wf, wt);
  count_launch();
}

void cnn_forward(cudaStream_t s, int B, int nx, int ny, const float* wf, const float* x, float* a1, float* a2,
                 float* y) {
  const dim3 g = tiles(nx, ny, B);
  k_conv3<4, 16><<<g, 256, 0, s>>>(nx, ny, x, wf, a1, 1, nullptr);
  k_conv3<16, 16><<<g, 256, 0, s>>>(nx, ny, a1, wf + 16 * 4 * 9, a2, 1, nullptr);
  k_conv3<16, 1><<<g, 256, 0, s>>>(nx, ny, a2, wf + 16 * 4 * 9 + 16 * 16 * 9, y, 0, nullptr);
  count_launch();
  count_launch();
  count_launch();
}

void cnn_backward(cudaStream_t s, int B, int nx, int ny, const float* wt, const float* x, const float* a1,
                  const float* a2, const float* y, const float* t, float* g3, float* g2, float* g1, double* tn2,
                  float* grad, double* loss) {
  const int npix = nx * ny;
  const dim3 g = tiles(nx, ny, B);
  const dim3 rb(std::min(64, (npix + 255) / 256), B);
  cudaMemsetAsync(tn2, 0, sizeof(double) * B, s);
  k_sample_norm2<<<rb, 256, 0, s>>>(npix, t, tn2);
  k_cnn_loss<<<rb, 256, 0, s>>>(B, npix, y, t, tn2, g3, loss);
  // layer 3: y = conv(a2, W3)
  k_conv3_wgrad<16, 1><<<g, 256, 0, s>>>(nx, ny, a2, g3, grad + 16 * 4 * 9 + 16 * 16 * 9);
  k_conv3<1, 16><<<g, 256, 0, s>>>(nx, ny, g3, wt + 16 * 4 * 9 + 16 * 16 * 9, g2, 0, a2);
  // layer 2: a2 = relu(conv(a1, W2))
  k_conv3_wgrad<16, 16><<<g, 256, 0, s>>>(nx, ny, a1, g2, grad + 16 * 4 * 9);
  k_conv3<16, 16><<<g, 256, 0, s>>>(nx, ny, g2, wt + 16 * 4 * 9, g1, 0, a1);
  // layer 1: a1 = relu(conv(x, W1))
  k_conv3_wgrad<4, 16><<<g, 256, 0, s>>>(nx, ny, x, g1, grad);
  for (int i = 0; i < 7; ++i) count_launch();
}

void cnn_adam(cudaStream_t s, float* w, float* grad, float* m, float* v, int step, float lr, float b1, float b2,
              float eps, void* params_bf16) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_cnn_adam<<<(CNN_NPARAM + 255) / 256, 256, 0, s>>>(CNN_NPARAM, w, grad, m, v, lr, b1, b2, eps, c1, c2,
                                                      static_cast<__nv_bfloat16*>(params_bf16));
  count_launch();
}

template <typename T>
void cnn_pack(cudaStream_t s, int n, int nb, const T* R, int ldr, const double* norms2, const float* feat,
              float* x) {
  const dim3 g(std::min(256, (n + 255) / 256), nb);
  k_cnn_pack<T><<<g, 256, 0, s>>>(n, nb, R, ldr, norms2, feat, x);
  count_launch();
}

template <typename T>
void cnn_unpack(cudaStream_t s, int n, int nb, const float* y, T* Tb, int ldt) {
  const dim3 g(std::min(256, (n + 255) / 256), nb);
  k_cnn_unpack<T><<<g, 256, 0, s>>>(n, nb, y, Tb, ldt);
  count_launch();
}

template void cnn_pack<double>(cudaStream_t, int, int, const double*, int, const double*, const float*, float*);
template void cnn_pack<float>(cudaStream_t, int, int, const float*, int, const double*, const float*, float*);
template void cnn_unpack<double>(cudaStream_t, int, int, const float*, double*, int);
template void cnn_unpack<float>(cudaStream_t, int, int, const float*, float*, int);

}  // namespace ph

// ===========================================================================
// C ABI (include/phsvds.h): forward, backward and Adam steps of the network.
// Workspace layout: tn2 (B doubles = 2B floats, first, so it is 8-byte
// aligned when the workspace is) | a1 | a2 (B*16*npix floats each) |
// g3 (B*npix) | g2 | g1 (B*16*npix each) | wf | wt (3024 each).
// ===========================================================================
namespace {
struct CnnWork {
  float *a1, *a2, *g3, *g2, *g1, *wf, *wt;
  double* tn2;
  CnnWork(float* w, int B, int npix) {
    const size_t P = (size_t)B * npix;
    tn2 = reinterpret_cast<double*>(w);
    a1 = w + 2 * (size_t)B;
    a2 = a1 + 16 * P;
    g3 = a2 + 16 * P;
    g2 = g3 + P;
    g1 = g2 + 16 * P;
    wf = g1 + 16 * P;
    wt = wf + ph::CNN_NPARAM;
  }
};
bool cnn_args_ok(int B, int nx, int ny) {
  return B >= 1 && nx >= 1 && ny >= 1 && (int64_t)B * nx * ny * 65 < (int64_t)1 << 34 && nx <= 65535 * ph::CNN_T &&
         ny <= 65535 * ph::CNN_T && B <= 65535;
}
phsvds_status cnn_status(phsvds_handle h) {
  const cudaError_t e = cudaGetLastError();
  (void)h;
  return e == cudaSuccess ? PHSVDS_OK : PHSVDS_ERR_CUDA;
}
}  // namespace

extern "C" phsvds_status phsvds_cnn_forward(phsvds_handle h, int batch, int nx, int ny, const void* params_bf16,
                                            const float* x, float* y, float* work) {
  if (!h || !params_bf16 || !x || !y || !work || ((uintptr_t)work & 7) || !cnn_args_ok(batch, nx, ny))
    return PHSVDS_ERR_INVALID;
  if (cudaSetDevice(ph::handle_device(h)) != cudaSuccess) return PHSVDS_ERR_CUDA;
  cudaStream_t s = ph::handle_stream(h);
  CnnWork w(work, batch, nx * ny);
  ph::cnn_weights(s, params_bf16, w.wf, w.wt);
  ph::cnn_forward(s, batch, nx, ny, w.wf, x, w.a1, w.a2, y);
  return cnn_status(h);
}

extern "C" phsvds_status phsvds_cnn_backward(phsvds_handle h, int batch, int nx, int ny, const void* params_bf16,
                                             const float* x, const float* y, const float* t, float* work,
                                             float* grad, double* loss) {
  if (!h || !params_bf16 || !x || !y || !t || !work || ((uintptr_t)work & 7) || !grad || !loss ||
      ((uintptr_t)loss & 7) || !cnn_args_ok(batch, nx, ny))
    return PHSVDS_ERR_INVALID;
  if (cudaSetDevice(ph::handle_device(h)) != cudaSuccess) return PHSVDS_ERR_CUDA;
  cudaStream_t s = ph::handle_stream(h);
  CnnWork w(work, batch, nx * ny);
  ph::cnn_backward(s, batch, nx, ny, w.wt, x, w.a1, w.a2, y, t, w.g3, w.g2, w.g1, w.tn2, grad, loss);
  return cnn_status(h);
}

extern "C" phsvds_status phsvds_cnn_adam(phsvds_handle h, float* master, float* grad, float* m, float* v, int step,
                                         float lr, float beta1, float beta2, float eps, void* params_bf16) {
  if (!h || !master || !grad || !m || !v || !params_bf16 || step < 1 || !(lr > 0.f)) return PHSVDS_ERR_INVALID;
  if (cudaSetDevice(ph::handle_device(h)) != cudaSuccess) return PHSVDS_ERR_CUDA;
  ph::cnn_adam(ph::handle_stream(h), master, grad, m, v, step, lr, beta1, beta2, eps, params_bf16);
  return cnn_status(h);
}
