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
// reduction accumulates per thread and per warp in FP32 and across warps and
// blocks in FP64.  The scalars of the b recurrences live on the device, so a step needs
// no host synchronisation and a run of steps replays as one CUDA graph.
#include "common.cuh"
#include "kernels.h"

namespace ph {

constexpr int JD_T = 256;

// V consecutive rows per thread, one 16-byte load (V = 4 for FP32, 2 for
// FP64) when n is a multiple of V, so that every column of a column-major
// block starts 16-byte aligned; else V = 1.
template <typename T, int V>
__device__ inline void ldv(const T* __restrict__ p, T (&r)[V]) {
  if constexpr (V == 1) {
    r[0] = *p;
  } else if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r[0] = t.x; r[1] = t.y;
  }
}
template <typename T, int V>
__device__ inline void stv(T* __restrict__ p, const T (&r)[V]) {
  if constexpr (V == 1)
    *p = r[0];
  else if constexpr (sizeof(T) == 4)
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  else
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}
// the wide form for element type T
template <typename T> constexpr int jd_wide() { return sizeof(T) == 4 ? 4 : 2; }


// ---- column reductions: acc[8 p + c] += sum_i a_p[c n + i] * b_p[c n + i] for
// the q columns of each of the NP pairs (a_p, b_p)
template <typename T, int NP>
struct DotPairs {
  const T* a[NP];
  const T* b[NP];
};

template <typename T, int NP, int V>
__global__ void __launch_bounds__(JD_T) k_col_dots(int n, int q, DotPairs<T, NP> pr, double* __restrict__ acc,
                                                   RedWs rw) {
  __shared__ double red[NP * 8][JD_T / 32];
  __shared__ double part[NP * 8];
  T s[NP][8];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) s[p][c] = T(0);
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= q) break;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        T a[V], b[V];
        ldv<T, V>(pr.a[p] + (size_t)c * n + i, a);
        ldv<T, V>(pr.b[p] + (size_t)c * n + i, b);
#pragma unroll
        for (int u = 0; u < V; ++u) s[p][c] = fma(a[u], b[u], s[p][c]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double v = warp_sum_wide<T>(s[p][c]);
      if (lane == 0) red[p * 8 + c][warp] = v;
    }
  __syncthreads();
  if (threadIdx.x < NP * 8) {
    double v = 0.0;
    if (threadIdx.x % 8 < q)
      for (int w = 0; w < JD_T / 32; ++w) v += red[threadIdx.x][w];
    part[threadIdx.x] = v;
  }
  __syncthreads();
  ordered_commit(part, NP * 8, acc, 0, nullptr, rw);
}

// The three column dots of a MINRES step, acc[c] += v_c^T Cv_c, acc[8 + c] +=
// v_c^T v_c, acc[16 + c] += x_c^T Cv_c: each array read once per column, and
// the columns guarded by a predicate rather than a loop exit, so that the
// loads of every column can be in flight together (one pass over a chunk of
// rows per thread leaves no later iteration to overlap them with).  Per
// column and per thread the sums run in the same order as k_col_dots<T, 3>.
template <typename T, int V>
__global__ void __launch_bounds__(JD_T) k_jd_dots3(int n, int q, const T* __restrict__ v, const T* __restrict__ X,
                                                   const T* __restrict__ Cv, double* __restrict__ acc, RedWs rw) {
  __shared__ double red[24][JD_T / 32];
  __shared__ double part[24];
  T s0[8], s1[8], s2[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) s0[c] = s1[c] = s2[c] = T(0);
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < q) {
        const size_t k = (size_t)c * n + i;
        T a[V], b[V], x[V];
        ldv<T, V>(v + k, a);
        ldv<T, V>(Cv + k, b);
        ldv<T, V>(X + k, x);
#pragma unroll
        for (int u = 0; u < V; ++u) {
          s0[c] = fma(a[u], b[u], s0[c]);
          s1[c] = fma(a[u], a[u], s1[c]);
          s2[c] = fma(x[u], b[u], s2[c]);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double w0 = warp_sum_wide<T>(s0[c]), w1 = warp_sum_wide<T>(s1[c]), w2 = warp_sum_wide<T>(s2[c]);
    if (lane == 0) red[c][warp] = w0, red[8 + c][warp] = w1, red[16 + c][warp] = w2;
  }
  __syncthreads();
  if (threadIdx.x < 24) {
    double t = 0.0;
    if (threadIdx.x % 8 < q)
      for (int w = 0; w < JD_T / 32; ++w) t += red[threadIdx.x][w];
    part[threadIdx.x] = t;
  }
  __syncthreads();
  ordered_commit(part, 24, acc, 0, nullptr, rw);
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

__global__ void k_jd_init(int q, const double* __restrict__ acc, double* __restrict__ sc) {
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
}

// r1 = r2 = R, v = R / beta1, s = w1 = w2 = 0
template <typename T, int V>
__global__ void __launch_bounds__(JD_T) k_jd_start(int n, int q, const T* __restrict__ R, T* __restrict__ r1,
                                                   T* __restrict__ r2, T* __restrict__ v, T* __restrict__ s,
                                                   T* __restrict__ w1, T* __restrict__ w2,
                                                   const double* __restrict__ sc) {
  __shared__ T sv[8];
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    sv[c] = (c < q && SC(JF_ACT, c) > 0.0) ? (T)(1.0 / SC(JF_BETA1, c)) : T(0);
  }
  __syncthreads();
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
    for (int c = 0; c < q; ++c) {
      const size_t k = (size_t)c * n + i;
      T r[V], z[V], vv[V];
      ldv<T, V>(R + k, r);
#pragma unroll
      for (int u = 0; u < V; ++u) z[u] = T(0), vv[u] = r[u] * sv[c];
      stv<T, V>(r1 + k, r);
      stv<T, V>(r2 + k, r);
      stv<T, V>(v + k, vv);
      stv<T, V>(s + k, z);
      stv<T, V>(w1 + k, z);
      stv<T, V>(w2 + k, z);
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

// y = C u - theta u - Xl (Xl^T C u) - x (x^T C u) - c1 r1 - c2 r2 (the projected,
// shifted operator and the Lanczos recurrence; u = v, and no x term when X is
// null); in the scaled form the operator part is multiplied by ds before the
// recurrence terms.  Then r1 <- r2, r2 <- y, and acc[24 + c] += ||y||^2.
// Columns already converged are left alone.  Each locked vector is loaded once
// per row group and applied to all columns.
template <typename T, int V>
__global__ void __launch_bounds__(JD_T) k_jd_lanczos(int n, int q, int nl, const T* __restrict__ Cv,
                                                     const T* __restrict__ v, const T* __restrict__ X,
                                                     const T* __restrict__ Xl, const double* __restrict__ theta,
                                                     const T* __restrict__ ds, T* __restrict__ r1,
                                                     T* __restrict__ r2, const double* __restrict__ sc,
                                                     double* __restrict__ acc, RedWs rw) {
  __shared__ T cf[8][4];               // theta, e, c1, c2 per column
  __shared__ T D[64 * 8];
  __shared__ double part[8];
  __shared__ double red[8][JD_T / 32];
  __shared__ int act[8];
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    const bool on = c < q && SC(JF_ACT, c) > 0.0;
    act[c] = on;
    cf[c][0] = on ? (T)theta[c] : T(0);
    cf[c][1] = (on && X) ? (T)acc[16 + c] : T(0);
    cf[c][2] = on ? (T)SC(JF_C1, c) : T(0);
    cf[c][3] = on ? (T)SC(JF_C2, c) : T(0);
  }
  for (int k = threadIdx.x; k < nl * 8; k += JD_T) {
    const int l = k % nl, c = k / nl;
    D[l * 8 + c] = (c < q && SC(JF_ACT, c) > 0.0) ? (T)acc[32 + l + c * nl] : T(0);
  }
  __syncthreads();
  T nrm[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) nrm[c] = T(0);
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
    T y[8][V];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < q) {
        const size_t k = (size_t)c * n + i;
        T a[V], b[V], d[V];
        ldv<T, V>(Cv + k, a);
        ldv<T, V>(v + k, b);
        if (X) {
          ldv<T, V>(X + k, d);
        } else {
#pragma unroll
          for (int u = 0; u < V; ++u) d[u] = T(0);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) y[c][u] = fma(-cf[c][1], d[u], fma(-cf[c][0], b[u], a[u]));
      }
    }
    // four locked vectors' loads in flight at a time (the sums per element
    // keep their order over l)
#pragma unroll 4
    for (int l = 0; l < nl; ++l) {
      T xl[V];
      ldv<T, V>(Xl + (size_t)l * n + i, xl);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < q) {
          const T dlc = D[l * 8 + c];
#pragma unroll
          for (int u = 0; u < V; ++u) y[c][u] = fma(-dlc, xl[u], y[c][u]);
        }
      }
    }
    if (ds) {
      T dd[V];
      ldv<T, V>(ds + i, dd);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < q) {
#pragma unroll
          for (int u = 0; u < V; ++u) y[c][u] *= dd[u];
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < q && act[c]) {
        const size_t k = (size_t)c * n + i;
        T a1[V], a2[V];
        ldv<T, V>(r1 + k, a1);
        ldv<T, V>(r2 + k, a2);
#pragma unroll
        for (int u = 0; u < V; ++u) {
          y[c][u] = fma(-cf[c][3], a2[u], fma(-cf[c][2], a1[u], y[c][u]));
          nrm[c] = fma(y[c][u], y[c][u], nrm[c]);
        }
        stv<T, V>(r1 + k, a2);
        stv<T, V>(r2 + k, y[c]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double t = warp_sum_wide<T>(nrm[c]);
    if (lane == 0) red[c][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
    if (threadIdx.x < q)
      for (int w = 0; w < JD_T / 32; ++w) t += red[threadIdx.x][w];
    part[threadIdx.x] = t;
  }
  __syncthreads();
  ordered_commit(part, 8, acc + 24, 0, nullptr, rw);
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
template <typename T, int V>
__global__ void __launch_bounds__(JD_T) k_jd_update(int n, int q, T* __restrict__ v, const T* __restrict__ r2,
                                                    T* __restrict__ w1, T* __restrict__ w2, T* __restrict__ s,
                                                    double* __restrict__ sc) {
  __shared__ T cf[8][5];
  __shared__ int on[8];
  if (threadIdx.x < 8) {
    const int c = threadIdx.x;
    const double act = c < q ? SC(JF_ACT, c) : 0.0;
    on[c] = act != 0.0;
    cf[c][0] = (T)SC(JF_OLDEPS, c);
    cf[c][1] = (T)SC(JF_DELTA, c);
    cf[c][2] = (T)(1.0 / SC(JF_GAMMA, c));
    cf[c][3] = (T)SC(JF_PHI, c);
    const double beta = SC(JF_BETA, c);
    cf[c][4] = (act > 0.0 && beta > 0.0) ? (T)(1.0 / beta) : T(0);
  }
  __syncthreads();
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= q || !on[c]) continue;
      const size_t k = (size_t)c * n + i;
      T a1[V], a2[V], vv[V], ss[V], rr[V], w[V];
      ldv<T, V>(w1 + k, a1);
      ldv<T, V>(w2 + k, a2);
      ldv<T, V>(v + k, vv);
      ldv<T, V>(s + k, ss);
      ldv<T, V>(r2 + k, rr);
#pragma unroll
      for (int u = 0; u < V; ++u) {
        w[u] = (vv[u] - cf[c][0] * a1[u] - cf[c][1] * a2[u]) * cf[c][2];
        ss[u] = fma(cf[c][3], w[u], ss[u]);
        vv[u] = rr[u] * cf[c][4];
      }
      stv<T, V>(w1 + k, a2);
      stv<T, V>(w2 + k, w);
      stv<T, V>(s + k, ss);
      stv<T, V>(v + k, vv);
    }
  }
}

// After the update of a stopping system (act = -1), mark it stopped.
__global__ void k_jd_retire(int q, double* __restrict__ sc) {
  const int c = threadIdx.x;
  if (c < q && SC(JF_ACT, c) < 0.0) SC(JF_ACT, c) = 0.0;
}
#undef SC

static int jd_grid(int n, int V) {
  int blocks = ceil_div(ceil_div(n, V), JD_T);
  return blocks > 152 * 8 ? 152 * 8 : (blocks < 1 ? 1 : blocks);
}
template <typename T> static int jd_vec(int n) { return n % jd_wide<T>() == 0 ? jd_wide<T>() : 1; }
template <typename T> static int jd_cls() { return sizeof(T) == 4 ? PROF_F32 + PROF_SMALL : PROF_SMALL; }

template <typename T>
void jd_colnorms(cudaStream_t s, int n, int q, const T* R, double* acc) {
  ProfScope ps(s, jd_cls<T>());
  DotPairs<T, 1> pr{{R}, {R}};
  const int V = jd_vec<T>(n), g = jd_grid(n, V);
  const RedWs rw = red_ws((size_t)g * 8);
  if (V > 1)
    k_col_dots<T, 1, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, pr, acc + 24, rw);
  else
    k_col_dots<T, 1, 1><<<g, JD_T, 0, s>>>(n, q, pr, acc + 24, rw);
  count_launch();
  reduce_partials(s, rw, g, 8, acc + 24, 0, nullptr);
}

template <typename T>
void jd_init(cudaStream_t s, int n, int q, const T* R, T* r1, T* r2, T* v, T* sol, T* w1, T* w2, const double* acc,
             double* sc) {
  ProfScope ps(s, jd_cls<T>());
  k_jd_init<<<1, 32, 0, s>>>(q, acc, sc); count_launch();
  const int V = jd_vec<T>(n), g = jd_grid(n, V);
  if (V > 1)
    k_jd_start<T, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, R, r1, r2, v, sol, w1, w2, sc);
  else
    k_jd_start<T, 1><<<g, JD_T, 0, s>>>(n, q, R, r1, r2, v, sol, w1, w2, sc);
  count_launch();
}

template <typename T>
void jd_dots(cudaStream_t s, int n, int q, const T* v, const T* X, const T* Cv, double* acc) {
  ProfScope ps(s, jd_cls<T>());
  const int V = jd_vec<T>(n), g = jd_grid(n, V);
  const RedWs rw = red_ws((size_t)g * 24);
  if (V > 1)
    k_jd_dots3<T, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, v, X, Cv, acc, rw);
  else
    k_jd_dots3<T, 1><<<g, JD_T, 0, s>>>(n, q, v, X, Cv, acc, rw);
  count_launch();
  reduce_partials(s, rw, g, 24, acc, 0, nullptr);
  count_work(jd_cls<T>(), 6.0 * n * q, (double)sizeof(T) * 3 * n * q);
}

template <typename T>
__global__ void k_jd_dscale(int n, const double* __restrict__ d, double guard, T* __restrict__ ds) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ds[i] = (T)(1.0 / sqrt(fmax(d[i], guard)));
}
template <typename T>
void jd_dscale(cudaStream_t s, int n, const double* d, double guard, T* ds) {
  if (n > 0) k_jd_dscale<T><<<ceil_div(n, 256), 256, 0, s>>>(n, d, guard, ds); count_launch();
}

template <typename T, int V>
__global__ void __launch_bounds__(JD_T) k_jd_rowscale(int n, int q, const T* __restrict__ ds, const T* __restrict__ X,
                                                      T* __restrict__ Y) {
  for (int i = (blockIdx.x * JD_T + threadIdx.x) * V; i < n; i += gridDim.x * JD_T * V) {
    T dd[V];
    ldv<T, V>(ds + i, dd);
    for (int c = 0; c < q; ++c) {
      T x[V];
      ldv<T, V>(X + (size_t)c * n + i, x);
#pragma unroll
      for (int u = 0; u < V; ++u) x[u] *= dd[u];
      stv<T, V>(Y + (size_t)c * n + i, x);
    }
  }
}
template <typename T>
void jd_rowscale(cudaStream_t s, int n, int q, const T* ds, const T* X, T* Y) {
  ProfScope ps(s, jd_cls<T>());
  if (n <= 0 || q <= 0) return;
  const int V = jd_vec<T>(n), g = jd_grid(n, V);
  if (V > 1)
    k_jd_rowscale<T, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, ds, X, Y);
  else
    k_jd_rowscale<T, 1><<<g, JD_T, 0, s>>>(n, q, ds, X, Y);
  count_launch();
}

template <typename T>
void jd_step(cudaStream_t s, int n, int q, int nl, const T* Cv, T* v, const T* u, const T* X, const T* Xl,
             const double* theta, const T* ds, T* r1, T* r2, T* w1, T* w2, T* sol, double* acc, double* sc,
             double tol) {
  ProfScope ps(s, jd_cls<T>());
  k_jd_coef<<<1, 32, 0, s>>>(q, acc, theta, sc); count_launch();
  const int V = jd_vec<T>(n), g = jd_grid(n, V);
  const RedWs rw = red_ws((size_t)g * 8);
  if (V > 1)
    k_jd_lanczos<T, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, nl, Cv, u, X, Xl, theta, ds, r1, r2, sc, acc, rw);
  else
    k_jd_lanczos<T, 1><<<g, JD_T, 0, s>>>(n, q, nl, Cv, u, X, Xl, theta, ds, r1, r2, sc, acc, rw);
  count_launch();
  reduce_partials(s, rw, g, 8, acc + 24, 0, nullptr);
  k_jd_givens<<<1, 32, 0, s>>>(q, acc, tol, sc); count_launch();
  if (V > 1)
    k_jd_update<T, jd_wide<T>()><<<g, JD_T, 0, s>>>(n, q, v, r2, w1, w2, sol, sc);
  else
    k_jd_update<T, 1><<<g, JD_T, 0, s>>>(n, q, v, r2, w1, w2, sol, sc);
  count_launch();
  k_jd_retire<<<1, 32, 0, s>>>(q, sc); count_launch();
  // the Lanczos pass reads Cv, v, x, r1, r2, Xl and writes r1, r2; the update
  // reads v, r2, w1, w2, s and writes w1, w2, s, v
  count_work(jd_cls<T>(), (2.0 * nl + 14.0) * n * q, (double)sizeof(T) * n * ((16.0 * q) + nl));
}

#define JD_INST(T)                                                                                                  \
  template void jd_colnorms<T>(cudaStream_t, int, int, const T*, double*);                                          \
  template void jd_init<T>(cudaStream_t, int, int, const T*, T*, T*, T*, T*, T*, T*, const double*, double*);       \
  template void jd_dots<T>(cudaStream_t, int, int, const T*, const T*, const T*, double*);                          \
  template void jd_dscale<T>(cudaStream_t, int, const double*, double, T*);                                         \
  template void jd_rowscale<T>(cudaStream_t, int, int, const T*, const T*, T*);                                     \
  template void jd_step<T>(cudaStream_t, int, int, int, const T*, T*, const T*, const T*, const T*, const double*,  \
                           const T*, T*, T*, T*, T*, T*, double*, double*, double);
JD_INST(float)
JD_INST(double)
#undef JD_INST

// ===========================================================================
// Stage 2 (Algorithm 2 with the JDQMR correction of Sec. 4): one correction
// equation (I - QQ^T)(B - mu I)(I - QQ^T) t = -(I - QQ^T) r at a time, FP64,
// Q = [locked vectors, their mirrors, x] (column-major N x nq).  MINRES as
// above (the scalar kernels are shared, with q = 1), plus the dynamic stop:
// after each step the updated vector z = x + t_k is scored by its
// eigen-residual eta_k = ||B z - rho z|| / ||z||, rho = z^T B z / z^T z, with
// B t_k carried by the same recurrence as t_k from the products the steps
// make (no extra product); the steps stop once eta_k < tol, once eta has not
// fallen below 0.9 of its best for `patience` steps, or at maxit, and the
// iterate with the smallest eta is kept.
// sc fields past the MINRES ones (index JF_NF * 8 + ...):
enum Jd2Field { J2_BEST = 0, J2_PREV_BEST, J2_SINCE, J2_COPY, J2_ETA, J2_STEPS, J2_NF };
#define S2(f) sc[JF_NF * 8 + (f)]
#define SC1(f) sc[(f) * 8]

// y = Bv - mu v - Q g - c1 r1 - c2 r2 (g = acc[32 ..] = Q^T Bv); r1 <- r2;
// r2 <- y; acc[24] += ||y||^2
__global__ void __launch_bounds__(JD_T) k_s2_lanczos(int64_t N, int nq, const double* __restrict__ Bv,
                                                     const double* __restrict__ v, const double* __restrict__ Q,
                                                     const double* __restrict__ mu, double* __restrict__ r1,
                                                     double* __restrict__ r2, const double* __restrict__ sc,
                                                     double* __restrict__ acc, RedWs rw) {
  __shared__ double g[65];
  __shared__ double red[JD_T / 32];
  __shared__ double part[1];
  if (SC1(JF_ACT) <= 0.0) {
    ordered_commit_zero(1, rw);
    return;
  }
  for (int l = threadIdx.x; l < nq; l += JD_T) g[l] = acc[32 + l];
  __syncthreads();
  const double m = mu[0], c1 = SC1(JF_C1), c2 = SC1(JF_C2);
  double nrm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)JD_T + threadIdx.x; i < N; i += (int64_t)gridDim.x * JD_T) {
    double y = fma(-m, v[i], Bv[i]);
    // four loads in flight at a time; the sum keeps its order over l
#pragma unroll 4
    for (int l = 0; l < nq; ++l) y = fma(-g[l], Q[(size_t)l * N + i], y);
    const double a2 = r2[i];
    y = fma(-c2, a2, fma(-c1, r1[i], y));
    r1[i] = a2;
    r2[i] = y;
    nrm = fma(y, y, nrm);
  }
  nrm = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < JD_T / 32; ++w) t += red[w];
    part[0] = t;
  }
  __syncthreads();
  ordered_commit(part, 1, acc + 24, 0, nullptr, rw);
}

// MINRES update of t and, by the same recurrence, of B t; v <- r2 / beta; then
// acc[160] += ||z||^2 and acc[161] += z^T B z for z = x + t, B z = Bx + Bt
__global__ void __launch_bounds__(JD_T) k_s2_update(int64_t N, double* __restrict__ v, const double* __restrict__ r2,
                                                    double* __restrict__ w1, double* __restrict__ w2,
                                                    double* __restrict__ t, const double* __restrict__ Bv,
                                                    double* __restrict__ Bw1, double* __restrict__ Bw2,
                                                    double* __restrict__ Bt, const double* __restrict__ x,
                                                    const double* __restrict__ Bx, const double* __restrict__ sc,
                                                    double* __restrict__ acc, RedWs rw) {
  __shared__ double red[2][JD_T / 32];
  __shared__ double part[2];
  const double act = SC1(JF_ACT);
  if (act == 0.0) {
    ordered_commit_zero(2, rw);
    return;
  }
  const double oldeps = SC1(JF_OLDEPS), delta = SC1(JF_DELTA), ig = 1.0 / SC1(JF_GAMMA), phi = SC1(JF_PHI);
  const double beta = SC1(JF_BETA);
  const double ib = (act > 0.0 && beta > 0.0) ? 1.0 / beta : 0.0;
  double zz = 0.0, zb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)JD_T + threadIdx.x; i < N; i += (int64_t)gridDim.x * JD_T) {
    const double a1 = w1[i], a2 = w2[i];
    const double w = (v[i] - oldeps * a1 - delta * a2) * ig;
    w1[i] = a2;
    w2[i] = w;
    const double tn = fma(phi, w, t[i]);
    t[i] = tn;
    const double b1 = Bw1[i], b2 = Bw2[i];
    const double bw = (Bv[i] - oldeps * b1 - delta * b2) * ig;
    Bw1[i] = b2;
    Bw2[i] = bw;
    const double btn = fma(phi, bw, Bt[i]);
    Bt[i] = btn;
    v[i] = r2[i] * ib;
    const double z = x[i] + tn, bz = Bx[i] + btn;
    zz = fma(z, z, zz);
    zb = fma(z, bz, zb);
  }
  zz = warp_sum(zz);
  zb = warp_sum(zb);
  if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = zz, red[1][threadIdx.x >> 5] = zb;
  __syncthreads();
  if (threadIdx.x < 2) {
    double u = 0.0;
    for (int w = 0; w < JD_T / 32; ++w) u += red[threadIdx.x][w];
    part[threadIdx.x] = u;
  }
  __syncthreads();
  ordered_commit(part, 2, acc + 160, 0, nullptr, rw);
}

// acc[162] += ||B z - rho z||^2, rho = acc[161] / acc[160] (a second pass: the
// short form ||Bz||^2 - rho^2 ||z||^2 would cancel far above the tolerance)
__global__ void __launch_bounds__(JD_T) k_s2_eta(int64_t N, const double* __restrict__ x, const double* __restrict__ t,
                                                 const double* __restrict__ Bx, const double* __restrict__ Bt,
                                                 const double* __restrict__ sc, double* __restrict__ acc,
                                                 RedWs rw) {
  __shared__ double red[JD_T / 32];
  __shared__ double part[1];
  if (SC1(JF_ACT) == 0.0) {
    ordered_commit_zero(1, rw);
    return;
  }
  const double rho = acc[160] > 0.0 ? acc[161] / acc[160] : 0.0;
  double e = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)JD_T + threadIdx.x; i < N; i += (int64_t)gridDim.x * JD_T) {
    const double d = (Bx[i] + Bt[i]) - rho * (x[i] + t[i]);
    e = fma(d, d, e);
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < JD_T / 32; ++w) u += red[w];
    part[0] = u;
  }
  __syncthreads();
  ordered_commit(part, 1, acc + 162, 0, nullptr, rw);
}

// The dynamic stop: best eta, the patience counter, the copy flag of this
// step's iterate; the system stops (act -1, retired after the copy) once
// best < tol, or patience steps pass without a 10% gain, or at maxit.
__global__ void k_s2_track(const double* __restrict__ acc, double tol, int patience, int maxit,
                           double* __restrict__ sc) {
  if (threadIdx.x != 0) return;
  S2(J2_COPY) = 0.0;
  const double act = SC1(JF_ACT);
  if (act == 0.0) return;
  const double eta = acc[160] > 0.0 ? sqrt(fmax(acc[162], 0.0) / acc[160]) : INFINITY;
  S2(J2_ETA) = eta;
  S2(J2_STEPS) += 1.0;
  const double best = S2(J2_BEST);
  if (eta < 0.9 * best) S2(J2_SINCE) = 0.0;
  else S2(J2_SINCE) += 1.0;
  if (eta < best) {
    S2(J2_BEST) = eta;
    S2(J2_COPY) = 1.0;
  }
  if (S2(J2_BEST) < tol || S2(J2_SINCE) >= patience || S2(J2_STEPS) >= maxit) SC1(JF_ACT) = -1.0;
}

__global__ void k_s2_copy(int64_t N, const double* __restrict__ t, double* __restrict__ tbest,
                          const double* __restrict__ sc) {
  if (S2(J2_COPY) == 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)JD_T + threadIdx.x; i < N; i += (int64_t)gridDim.x * JD_T) tbest[i] = t[i];
}

__global__ void k_s2_init(double* __restrict__ sc) {
  if (threadIdx.x != 0) return;
  S2(J2_BEST) = INFINITY;
  S2(J2_SINCE) = 0.0;
  S2(J2_COPY) = 0.0;
  S2(J2_ETA) = INFINITY;
  S2(J2_STEPS) = 0.0;
}
#undef S2
#undef SC1

static int s2_grid(int64_t N) {
  int64_t b = (N + JD_T - 1) / JD_T;
  return (int)(b > 152 * 4 ? 152 * 4 : (b < 1 ? 1 : b));
}

// v = R / beta1 (zero when the system does not iterate)
__global__ void k_s2_first(int64_t N, const double* __restrict__ R, double* __restrict__ v,
                           const double* __restrict__ sc) {
  const double b1 = sc[JF_BETA1 * 8];
  const double f = (sc[JF_ACT * 8] > 0.0 && b1 > 0.0) ? 1.0 / b1 : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)JD_T + threadIdx.x; i < N; i += (int64_t)gridDim.x * JD_T) v[i] = R[i] * f;
}

void s2_start(cudaStream_t s, int64_t N, const double* R, double* r1, double* r2, double* v, double* t, double* w1,
              double* w2, double* Bt, double* Bw1, double* Bw2, double* acc, double* sc) {
  ProfScope ps(s, PROF_SMALL);
  cudaMemsetAsync(acc, 0, sizeof(double) * 256, s);
  dot_accum(s, N, R, R, acc + 24);
  k_jd_init<<<1, 32, 0, s>>>(1, acc, sc); count_launch();
  k_s2_init<<<1, 32, 0, s>>>(sc); count_launch();
  cudaMemcpyAsync(r1, R, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(r2, R, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  k_s2_first<<<s2_grid(N), JD_T, 0, s>>>(N, R, v, sc); count_launch();
  for (double* z : {t, w1, w2, Bt, Bw1, Bw2}) cudaMemsetAsync(z, 0, sizeof(double) * N, s);
}

// one MINRES step after the product Bv = B v and the reductions acc[0] = v^T Bv,
// acc[8] = v^T v, acc[32 ..] = Q^T Bv (acc[24], acc[160..163) zeroed)
void s2_step(cudaStream_t s, int64_t N, int nq, const double* Bv, double* v, const double* Q, const double* mu,
             double* r1, double* r2, double* w1, double* w2, double* t, double* Bw1, double* Bw2, double* Bt,
             const double* x, const double* Bx, double* tbest, double* acc, double* sc, double eta_tol, int patience,
             int maxit) {
  ProfScope ps(s, PROF_SMALL);
  const int g = s2_grid(N);
  k_jd_coef<<<1, 32, 0, s>>>(1, acc, mu, sc); count_launch();
  const RedWs rw1 = red_ws((size_t)g), rw2 = red_ws((size_t)g * 2);
  k_s2_lanczos<<<g, JD_T, 0, s>>>(N, nq, Bv, v, Q, mu, r1, r2, sc, acc, rw1); count_launch();
  reduce_partials(s, rw1, g, 1, acc + 24, 0, nullptr);
  k_jd_givens<<<1, 32, 0, s>>>(1, acc, 1e-15, sc); count_launch();
  k_s2_update<<<g, JD_T, 0, s>>>(N, v, r2, w1, w2, t, Bv, Bw1, Bw2, Bt, x, Bx, sc, acc, rw2); count_launch();
  reduce_partials(s, rw2, g, 2, acc + 160, 0, nullptr);
  k_s2_eta<<<g, JD_T, 0, s>>>(N, x, t, Bx, Bt, sc, acc, rw1); count_launch();
  reduce_partials(s, rw1, g, 1, acc + 162, 0, nullptr);
  k_s2_track<<<1, 32, 0, s>>>(acc, eta_tol, patience, maxit, sc); count_launch();
  k_s2_copy<<<g, JD_T, 0, s>>>(N, t, tbest, sc); count_launch();
  k_jd_retire<<<1, 32, 0, s>>>(1, sc); count_launch();
  count_work(PROF_SMALL, 2.0 * N * (nq + 16), 8.0 * N * (nq + 22));
}

}  // namespace ph
