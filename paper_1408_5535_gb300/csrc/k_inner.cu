// Inner solves of the Jacobi-Davidson correction equation in FP32.
//
// The JDQMR form of the method (Sec. 4) expands the basis by an approximate
// solution t of the correction equation
//     (I - Q Q^T) (C - theta I) (I - Q Q^T) t = r,   Q = [locked vectors, x],
// for a Ritz pair (theta, x) with residual r, instead of by r itself.  Here the
// equation is solved for b targets at once (each with its own theta and x) by
// the minimum-residual Krylov method for symmetric operators (MINRES, Paige
// and Saunders 1975: Lanczos three-term recurrence plus a QR factorisation of
// the tridiagonal by Givens rotations), in FP32 with the FP32 copy of A: on
// GB300 an FP32 product with C costs about a fifth of an FP64 one, and the
// outer Rayleigh-Ritz step, which alone sets the attainable accuracy, stays
// in FP64.
//
// Vectors are FP32, column-major n x b (leading dimension n); every
// reduction accumulates per thread in FP32 and across threads and blocks in
// FP64.  The scalars of the b recurrences live on the device, so a step needs
// no host synchronisation and a run of steps replays as one CUDA graph.
#include "common.cuh"
#include "kernels.h"

namespace ph {

constexpr int JD_T = 256;

// ---- column reductions: acc[8 p + c] += sum_i a_p[c n + i] * b_p[c n + i] for
// the q columns of each of the NP pairs (a_p, b_p)
template <int NP>
struct DotPairs {
  const float* a[NP];
  const float* b[NP];
};

template <int NP>
__global__ void __launch_bounds__(JD_T) k_col_dots(int n, int q, DotPairs<NP> pr, double* __restrict__ acc) {
  __shared__ double red[NP * 8][JD_T / 32];
  float s[NP][8];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) s[p][c] = 0.f;
  for (int i = blockIdx.x * JD_T + threadIdx.x; i < n; i += gridDim.x * JD_T) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float* a = pr.a[p];
      const float* b = pr.b[p];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < q) s[p][c] = fmaf(a[(size_t)c * n + i], b[(size_t)c * n + i], s[p][c]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double v = warp_sum((double)s[p][c]);
      if (lane == 0) red[p * 8 + c][warp] = v;
    }
  __syncthreads();
  if (threadIdx.x < NP * 8) {
    const int p = threadIdx.x / 8, c = threadIdx.x % 8;
    if (c < q) {
      double v = 0.0;
      for (int w = 0; w < JD_T / 32; ++w) v += red[threadIdx.x][w];
      atomicAdd(&acc[p * 8 + c], v);
    }
  }
}

// ---- MINRES state of the b systems: sc[field * 8 + c]
enum JdField {
  JF_BETA1 = 0, JF_BETA, JF_OLDB, JF_DBAR, JF_EPSLN, JF_PHIBAR, JF_CS, JF_SN, JF_PHI, JF_GAMMA, JF_DELTA,
  JF_OLDEPS, JF_ALFA, JF_C1, JF_C2, JF_ACT, JF_STEP, JF_NF
};
#define SC(f, c) sc[(f) * 8 + (c)]

// acc layout (FP64, zeroed before each reduction): [0,8) v^T C v, [8,16) v^T v,
// [16,24) x^T C v, [24,32) ||y||^2, [32, 32 + 8 nl) the projections Xl^T C v
// (nl x b, column-major with leading dimension nl).

__global__ void k_jd_init(int q, const double* __restrict__ acc, double tol, double* __restrict__ sc) {
  const int c = threadIdx.x;
  if (c >= 8) return;
  const double b1 = c < q ? sqrt(fmax(acc[24 + c], 0.0)) : 0.0;
  SC(JF_BETA1, c) = b1;
  SC(JF_BETA, c) = b1;
  SC(JF_OLDB, c) = 0.0;
  SC(JF_DBAR, c) = 0.0;
  SC(JF_EPSLN, c) = 0.0;
  SC(JF_PHIBAR, c) = b1;
  SC(JF_CS, c) = -1.0;
  SC(JF_SN, c) = 0.0;
  SC(JF_PHI, c) = 0.0;
  SC(JF_GAMMA, c) = 1.0;
  SC(JF_DELTA, c) = 0.0;
  SC(JF_OLDEPS, c) = 0.0;
  SC(JF_ALFA, c) = 0.0;
  SC(JF_C1, c) = 0.0;
  SC(JF_C2, c) = 0.0;
  SC(JF_ACT, c) = (c < q && b1 > 0.0 && isfinite(b1)) ? 1.0 : 0.0;
  SC(JF_STEP, c) = 0.0;
  (void)tol;
}

// r1 = r2 = R, v = R / beta1, s = w1 = w2 = 0
__global__ void k_jd_start(int n, int q, const float* __restrict__ R, float* __restrict__ r1, float* __restrict__ r2,
                           float* __restrict__ v, float* __restrict__ s, float* __restrict__ w1,
                           float* __restrict__ w2, const double* __restrict__ sc) {
  for (int i = blockIdx.x * JD_T + threadIdx.x; i < n; i += gridDim.x * JD_T) {
    for (int c = 0; c < q; ++c) {
      const size_t k = (size_t)c * n + i;
      const float r = R[k];
      const double b1 = SC(JF_BETA1, c);
      r1[k] = r;
      r2[k] = r;
      v[k] = SC(JF_ACT, c) > 0.0 ? (float)((double)r / b1) : 0.f;
      s[k] = 0.f;
      w1[k] = 0.f;
      w2[k] = 0.f;
    }
  }
}

// Lanczos coefficients of this step: alfa = v^T (C - theta) v, and the
// multipliers of r1 (beta / oldbeta, from the second step on) and r2 (alfa / beta).
__global__ void k_jd_coef(int q, const double* __restrict__ acc, const double* __restrict__ theta,
                          double* __restrict__ sc) {
  const int c = threadIdx.x;
  if (c >= q || SC(JF_ACT, c) == 0.0) return;
  const double alfa = acc[c] - theta[c] * acc[8 + c];
  const double beta = SC(JF_BETA, c), oldb = SC(JF_OLDB, c);
  SC(JF_ALFA, c) = alfa;
  SC(JF_C1, c) = (SC(JF_STEP, c) > 0.0 && oldb > 0.0) ? beta / oldb : 0.0;
  SC(JF_C2, c) = alfa / beta;
}

// y = C v - theta v - Xl (Xl^T C v) - x (x^T C v) - c1 r1 - c2 r2 (the projected,
// shifted operator and the Lanczos recurrence); then r1 <- r2, r2 <- y, and
// acc[24 + c] += ||y||^2.  Columns already converged are left alone.
template <int NL>
__global__ void __launch_bounds__(JD_T) k_jd_lanczos(int n, int q, int nl, const float* __restrict__ Cv,
                                                     const float* __restrict__ v, const float* __restrict__ X,
                                                     const float* __restrict__ Xl, const double* __restrict__ theta,
                                                     float* __restrict__ r1, float* __restrict__ r2,
                                                     const double* __restrict__ sc, double* __restrict__ acc) {
  __shared__ float cf[8][4];           // theta, e, c1, c2 per column
  __shared__ float D[NL > 0 ? NL * 8 : 1];
  __shared__ double red[8][JD_T / 32];
  __shared__ int act[8];
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    const bool on = c < q && SC(JF_ACT, c) > 0.0;
    act[c] = on;
    cf[c][0] = on ? (float)theta[c] : 0.f;
    cf[c][1] = on ? (float)acc[16 + c] : 0.f;
    cf[c][2] = on ? (float)SC(JF_C1, c) : 0.f;
    cf[c][3] = on ? (float)SC(JF_C2, c) : 0.f;
  }
  for (int k = threadIdx.x; k < nl * 8; k += JD_T) {
    const int l = k % nl, c = k / nl;
    D[k] = (c < q && SC(JF_ACT, c) > 0.0) ? (float)acc[32 + l + c * nl] : 0.f;
  }
  __syncthreads();
  float nrm[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) nrm[c] = 0.f;
  for (int i = blockIdx.x * JD_T + threadIdx.x; i < n; i += gridDim.x * JD_T) {
    float xl[NL > 0 ? NL : 1];
#pragma unroll
    for (int l = 0; l < NL; ++l) xl[l] = l < nl ? Xl[(size_t)l * n + i] : 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= q || !act[c]) continue;
      const size_t k = (size_t)c * n + i;
      float y = fmaf(-cf[c][0], v[k], Cv[k]);
      y = fmaf(-cf[c][1], X[k], y);
#pragma unroll
      for (int l = 0; l < NL; ++l)
        if (l < nl) y = fmaf(-D[l + c * nl], xl[l], y);
      const float a2 = r2[k];
      y = fmaf(-cf[c][2], r1[k], y);
      y = fmaf(-cf[c][3], a2, y);
      r1[k] = a2;
      r2[k] = y;
      nrm[c] = fmaf(y, y, nrm[c]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double t = warp_sum((double)nrm[c]);
    if (lane == 0) red[c][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < q) {
    double t = 0.0;
    for (int w = 0; w < JD_T / 32; ++w) t += red[threadIdx.x][w];
    atomicAdd(&acc[24 + threadIdx.x], t);
  }
}

// The Givens step of MINRES for each active system: the previous rotation
// applied to the new column of the tridiagonal, the next rotation, and the
// step length phi of the solution update; the system stops once its residual
// estimate phibar falls to tol * beta1 (or the Lanczos vector vanishes).
__global__ void k_jd_givens(int q, const double* __restrict__ acc, double tol, double* __restrict__ sc) {
  const int c = threadIdx.x;
  if (c >= q) return;
  if (SC(JF_ACT, c) == 0.0) {
    SC(JF_PHI, c) = 0.0;
    return;
  }
  const double alfa = SC(JF_ALFA, c);
  const double oldb = SC(JF_BETA, c);
  const double beta = sqrt(fmax(acc[24 + c], 0.0));
  const double cs = SC(JF_CS, c), sn = SC(JF_SN, c), dbar = SC(JF_DBAR, c);
  const double oldeps = SC(JF_EPSLN, c);
  const double delta = cs * dbar + sn * alfa;
  const double gbar = sn * dbar - cs * alfa;
  const double epsln = sn * beta;
  const double dbar2 = -cs * beta;
  const double gamma = fmax(sqrt(gbar * gbar + beta * beta), 1e-300);
  const double cs2 = gbar / gamma, sn2 = beta / gamma;
  const double phibar = SC(JF_PHIBAR, c);
  SC(JF_OLDB, c) = oldb;
  SC(JF_BETA, c) = beta;
  SC(JF_OLDEPS, c) = oldeps;
  SC(JF_DELTA, c) = delta;
  SC(JF_EPSLN, c) = epsln;
  SC(JF_DBAR, c) = dbar2;
  SC(JF_GAMMA, c) = gamma;
  SC(JF_CS, c) = cs2;
  SC(JF_SN, c) = sn2;
  SC(JF_PHI, c) = cs2 * phibar;
  SC(JF_PHIBAR, c) = sn2 * phibar;
  SC(JF_STEP, c) += 1.0;
  const double b1 = SC(JF_BETA1, c);
  const bool done = !(sn2 * fabs(phibar) > tol * b1) || !(beta > 1e-30 * b1);
  if (done) SC(JF_ACT, c) = -1.0;   // -1: this step's update still applies, then stop
}

// w = (v - oldeps w1 - delta w2) / gamma;  w1 <- w2;  w2 <- w;  s += phi w;
// v <- r2 / beta for the next step.
__global__ void __launch_bounds__(JD_T) k_jd_update(int n, int q, float* __restrict__ v, const float* __restrict__ r2,
                                                    float* __restrict__ w1, float* __restrict__ w2,
                                                    float* __restrict__ s, double* __restrict__ sc) {
  __shared__ float cf[8][5];
  __shared__ int on[8];
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    const double act = c < q ? SC(JF_ACT, c) : 0.0;
    on[c] = act != 0.0;
    cf[c][0] = (float)SC(JF_OLDEPS, c);
    cf[c][1] = (float)SC(JF_DELTA, c);
    cf[c][2] = (float)(1.0 / SC(JF_GAMMA, c));
    cf[c][3] = (float)SC(JF_PHI, c);
    const double beta = SC(JF_BETA, c);
    cf[c][4] = (act > 0.0 && beta > 0.0) ? (float)(1.0 / beta) : 0.f;
  }
  __syncthreads();
  for (int i = blockIdx.x * JD_T + threadIdx.x; i < n; i += gridDim.x * JD_T) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= q || !on[c]) continue;
      const size_t k = (size_t)c * n + i;
      const float a1 = w1[k], a2 = w2[k];
      const float w = (v[k] - cf[c][0] * a1 - cf[c][1] * a2) * cf[c][2];
      w1[k] = a2;
      w2[k] = w;
      s[k] = fmaf(cf[c][3], w, s[k]);
      v[k] = r2[k] * cf[c][4];
    }
  }
}

// After the update of a stopping system (act = -1), mark it stopped.
__global__ void k_jd_retire(int q, double* __restrict__ sc) {
  const int c = threadIdx.x;
  if (c < q && SC(JF_ACT, c) < 0.0) SC(JF_ACT, c) = 0.0;
}
#undef SC

static int jd_grid(int n) {
  int blocks = ceil_div(n, JD_T);
  return blocks > 152 * 8 ? 152 * 8 : (blocks < 1 ? 1 : blocks);
}

void jd_colnorms(cudaStream_t s, int n, int q, const float* R, double* acc) {
  ProfScope ps(s, PROF_F32 + PROF_SMALL);
  DotPairs<1> pr{{R}, {R}};
  k_col_dots<1><<<jd_grid(n), JD_T, 0, s>>>(n, q, pr, acc + 24); count_launch();
}

void jd_init(cudaStream_t s, int n, int q, const float* R, float* r1, float* r2, float* v, float* sol, float* w1,
             float* w2, const double* acc, double* sc) {
  ProfScope ps(s, PROF_F32 + PROF_SMALL);
  k_jd_init<<<1, 32, 0, s>>>(q, acc, 0.0, sc); count_launch();
  k_jd_start<<<jd_grid(n), JD_T, 0, s>>>(n, q, R, r1, r2, v, sol, w1, w2, sc); count_launch();
}

void jd_dots(cudaStream_t s, int n, int q, const float* v, const float* X, const float* Cv, double* acc) {
  ProfScope ps(s, PROF_F32 + PROF_SMALL);
  DotPairs<3> pr{{v, v, X}, {Cv, v, Cv}};
  k_col_dots<3><<<jd_grid(n), JD_T, 0, s>>>(n, q, pr, acc); count_launch();
  count_work(PROF_F32 + PROF_SMALL, 6.0 * n * q, 4.0 * 3 * n * q);
}

void jd_step(cudaStream_t s, int n, int q, int nl, const float* Cv, float* v, const float* X, const float* Xl,
             const double* theta, float* r1, float* r2, float* w1, float* w2, float* sol, double* acc, double* sc,
             double tol) {
  ProfScope ps(s, PROF_F32 + PROF_SMALL);
  k_jd_coef<<<1, 32, 0, s>>>(q, acc, theta, sc); count_launch();
  const int g = jd_grid(n);
  if (nl == 0)
    k_jd_lanczos<0><<<g, JD_T, 0, s>>>(n, q, nl, Cv, v, X, Xl, theta, r1, r2, sc, acc);
  else if (nl <= 8)
    k_jd_lanczos<8><<<g, JD_T, 0, s>>>(n, q, nl, Cv, v, X, Xl, theta, r1, r2, sc, acc);
  else if (nl <= 16)
    k_jd_lanczos<16><<<g, JD_T, 0, s>>>(n, q, nl, Cv, v, X, Xl, theta, r1, r2, sc, acc);
  else if (nl <= 32)
    k_jd_lanczos<32><<<g, JD_T, 0, s>>>(n, q, nl, Cv, v, X, Xl, theta, r1, r2, sc, acc);
  else
    k_jd_lanczos<64><<<g, JD_T, 0, s>>>(n, q, nl, Cv, v, X, Xl, theta, r1, r2, sc, acc);
  count_launch();
  k_jd_givens<<<1, 32, 0, s>>>(q, acc, tol, sc); count_launch();
  k_jd_update<<<g, JD_T, 0, s>>>(n, q, v, r2, w1, w2, sol, sc); count_launch();
  k_jd_retire<<<1, 32, 0, s>>>(q, sc); count_launch();
  // the Lanczos pass reads Cv, v, x, r1, r2, Xl and writes r1, r2; the update
  // reads v, r2, w1, w2, s and writes w1, w2, s, v
  count_work(PROF_F32 + PROF_SMALL, (2.0 * nl + 14.0) * n * q, 4.0 * n * ((16.0 * q) + nl));
}

}  // namespace ph
