// Kernels for the projected (small) problems of PHSVDS:
//  * cyclic two-sided Jacobi eigensolvers for the Rayleigh-Ritz matrix
//    H = V^T W (the projected problem of GD+k in stage 1, Algorithm 2 step 7
//    in stage 2), run in a warm frame (the working matrix A = S^T H S and the
//    accumulated rotation S are kept between outer iterations): an FP32 pass
//    followed by an FP64 clean-up of the target pairs, or FP64 in one CTA or
//    over an 8-CTA cluster;
//  * the refined vector of stage 2 (Algorithm 2 step 8): the smallest right
//    singular vector of the triangular factor R by inverse iteration, and the
//    whole one-sided (Hestenes) Jacobi SVD of R as an entry point;
//  * Cholesky of a block Gram matrix (CholQR of the new block), the restart /
//    locking transform builder and small gathers.
// Small matrices are column-major with a leading dimension ld (<= 64).
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace ph {

constexpr int SM_MAXJ = 64;
constexpr int SM_THREADS = 256;

// Round-robin (circle) pairing of jj (even) indices: round r, pair k.
__device__ inline void rr_pair(int jj, int r, int k, int& p, int& q) {
  const int m = jj - 1;
  int a, b;
  if (k == 0) {
    a = r % m;
    b = m;
  } else {
    a = (r + k) % m;
    b = (r - k + m) % m;
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Rotation of the pair (p, q) that (nearly) annihilates a_pq.  The angle is
// computed in FP32 from the entries scaled by 1/scale (FP64 division and square
// root are long dependent chains on GB300's FP64 pipe); c and s are then made
// orthonormal in FP64, so every rotation is exact to FP64 rounding while a_pq
// shrinks by ~1e-7 per rotation (the next sweep removes the rest).
// c = x^(-1/2), x = 1 + t^2, from the FP32 estimate y by one Halley step,
// y (15 - 10 h + 3 h^2) / 8 with h = x y^2 (cubic convergence: 24 bits to
// well past 53), then s = t c.
__device__ inline void rot_params(double app, double aqq, double apq, double inv_scale, double& c, double& s_) {
  const float fpp = (float)(app * inv_scale), fqq = (float)(aqq * inv_scale), fpq = (float)(apq * inv_scale);
  const float ftau = (fqq - fpp) / (2.0f * fpq);
  const float ft = copysignf(1.0f, ftau) / (fabsf(ftau) + sqrtf(1.0f + ftau * ftau));
  const double t = (double)ft;
  const double x = fma(t, t, 1.0);
  const double y = (double)rsqrtf((float)x);
  const double h = x * (y * y);
  const double q = y * 0.125;
  const double cc = q * fma(h, fma(h, 3.0, -10.0), 15.0);
  c = cc;
  s_ = t * cc;
}

// ---------------------------------------------------------------------------
// Two-sided cyclic Jacobi.  A rotation is applied to pair (p, q) when
// |a_pq| > thr, thr = tol * max_i |a_ii| (absolute accuracy tol * ||H||).
// Each round rotates up to jj/2 disjoint pairs at once; the update of A is
// done per 2 x 2 block (pair k rows, pair l columns), so one round needs a
// single barrier after the rotation parameters and one after the update.
// ---------------------------------------------------------------------------
// R = double: the FP64 solver (in place on H, S <- S J).  R = float: the bulk
// pass of the mixed-precision solver -- H is read and left unchanged, and S
// receives the FP32 rotation J alone (S_in is ignored), converted to FP64.
template <typename R>
__global__ void __launch_bounds__(SM_THREADS) k_jacobi_eig(int j, double* H, int ldh, double* S, int lds,
                                                           double* theta, double tol, int max_sweeps,
                                                           int* sweeps_out, double tol_loose, int ntarget,
                                                           int tmode, double tshift, int* rot_out) {
  extern __shared__ __align__(16) double dsm[];
  R* A = reinterpret_cast<R*>(dsm);                              // [SM_MAXJ * (SM_MAXJ + 1)]
  R* Sm = A + SM_MAXJ * (SM_MAXJ + 1);     // [SM_MAXJ * (SM_MAXJ + 1)]
  __shared__ R cs[SM_MAXJ / 2], sn[SM_MAXJ / 2], tt[SM_MAXJ / 2];
  __shared__ int pp[SM_MAXJ / 2], qq[SM_MAXJ / 2], rot[SM_MAXJ / 2];
  __shared__ R scale_s;
  constexpr bool F64 = sizeof(R) == 8;
  const int tid = threadIdx.x;
  const int LA = SM_MAXJ + 1;
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    A[r + c * LA] = (R)H[r + (size_t)c * ldh];
    Sm[r + c * LA] = F64 ? (R)S[r + (size_t)c * lds] : (R)(r == c ? 1 : 0);
  }
  __syncthreads();
  if (tid < 32) {
    R mx = 0;
    for (int i = tid; i < j; i += 32) mx = fmax(mx, fabs(A[i + i * LA]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) scale_s = mx;
  }
  __syncthreads();
  R mxoff = 0;
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    if (r != c) mxoff = fmax(mxoff, fabs(A[r + c * LA]));
  }
  // the scale must cover an all-zero diagonal (e.g. the augmented matrix)
  for (int o = 16; o > 0; o >>= 1) mxoff = fmax(mxoff, __shfl_xor_sync(0xffffffffu, mxoff, o));
  __shared__ R wmx[SM_THREADS / 32];
  if ((tid & 31) == 0) wmx[tid >> 5] = mxoff;
  __syncthreads();
  if (tid == 0) {
    R m2 = 0;
    for (int w = 0; w < SM_THREADS / 32; ++w) m2 = fmax(m2, wmx[w]);
    scale_s = fmax(scale_s, m2);
  }
  __syncthreads();
  const R thr_t = (R)(tol * (double)scale_s);
  const double inv_scale = (double)scale_s > 0.0 ? 1.0 / (double)scale_s : 1.0;                                  // pairs touching a target
  // pairs not touching a target rotate when |a_pq| > tol_loose sqrt|a_pp a_qq|
  // (relative, never below the absolute threshold); ntarget = 0: absolute everywhere
  const R rel = (R)(ntarget > 0 ? tol_loose : 0.0);
  const int jj = j + (j & 1);
  const int np = jj / 2;
  // targets: the ntarget smallest (tmode 0), largest (1) or closest to tshift
  // (2) diagonal entries, re-ranked at the start of every sweep
  __shared__ unsigned char is_t[SM_MAXJ];
  auto need = [&](int p, int q, R apq) -> bool {
    if (is_t[p] | is_t[q]) return fabs(apq) > thr_t;
    if (rel == (R)0) return fabs(apq) > thr_t;
    const float r2 = (float)rel * sqrtf(fabsf((float)A[p + p * LA] * (float)A[q + q * LA]));
    return fabs(apq) > ((R)r2 > thr_t ? (R)r2 : thr_t);
  };
  int sweep = 0;
  int nrot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid < j) {
      int r = 1;
      if (ntarget > 0) {
        auto key = [&](int t2) {
          const double d = (double)A[t2 + t2 * LA];
          return tmode == 0 ? d : (tmode == 1 ? -d : fabs(d - tshift));
        };
        const double ki = key(tid);
        int rank = 0;
        for (int t2 = 0; t2 < j; ++t2) {
          const double kt = key(t2);
          if (kt < ki || (kt == ki && t2 < tid)) ++rank;
        }
        r = rank < ntarget;
      }
      is_t[tid] = (unsigned char)r;
    }
    __syncthreads();
    int any = 0;
    for (int e = tid; e < j * j; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      if (r < c && need(r, c, A[r + c * LA])) any = 1;
    }
    if (!__syncthreads_or(any)) break;
    for (int round = 0; round < jj - 1; ++round) {
      int mine = 0;
      if (tid < np) {
        int p, q;
        rr_pair(jj, round, tid, p, q);
        pp[tid] = p;
        qq[tid] = q;
        int r = 0;
        if (q < j) {
          const R apq = A[p + q * LA];
          if (need(p, q, apq)) {
            if constexpr (F64) {
              double c, sv;
              rot_params(A[p + p * LA], A[q + q * LA], apq, inv_scale, c, sv);
              cs[tid] = c;
              sn[tid] = sv;
            } else {
              const R tau = (A[q + q * LA] - A[p + p * LA]) / ((R)2 * apq);
              const R t = (tau >= (R)0 ? (R)1 : (R)-1) / (fabs(tau) + sqrt((R)1 + tau * tau));
              const R c = (R)1 / sqrt((R)1 + t * t);
              cs[tid] = c;
              sn[tid] = t * c;
            }
            r = 1;
          }
        }
        rot[tid] = r;
        mine = r;
      }
      if (!__syncthreads_or(mine)) continue;
      if (tid == 0) {
        int cnt = 0;
        for (int k2 = 0; k2 < np; ++k2) cnt += rot[k2];
        nrot += cnt;
      }
      // 2 x 2 blocks (k, l): rows of pair k, columns of pair l
      for (int it = tid; it < np * np; it += SM_THREADS) {
        const int k = it / np, l = it % np;
        const int rk = rot[k], rl = rot[l];
        if (!rk && !rl) continue;
        const int pk = pp[k], qk = qq[k], pl = pp[l], ql = qq[l];
        if (k == l) {
          if (qk < j) {  // full 2 x 2 update J^T B J (the angle is not exact)
            const R c = cs[k], sv = sn[k];
            const R app = A[pk + pk * LA], aqq = A[qk + qk * LA], apq = A[pk + qk * LA];
            const R r00 = c * app - sv * apq, r01 = c * apq - sv * aqq;
            const R r10 = sv * app + c * apq, r11 = sv * apq + c * aqq;
            const R n00 = c * r00 - sv * r01, n11 = sv * r10 + c * r11;
            const R n01 = (sv * r00 + c * r01 + c * r10 - sv * r11) * (R)0.5;
            A[pk + pk * LA] = n00;
            A[qk + qk * LA] = n11;
            A[pk + qk * LA] = n01;
            A[qk + pk * LA] = n01;
          }
          continue;
        }
        const R ck = rk ? cs[k] : (R)1, sk = rk ? sn[k] : (R)0;
        const R cl = rl ? cs[l] : (R)1, sl = rl ? sn[l] : (R)0;
        const bool vqk = qk < j, vql = ql < j;
        const R b00 = A[pk + pl * LA];
        const R b01 = vql ? A[pk + ql * LA] : (R)0;
        const R b10 = vqk ? A[qk + pl * LA] : (R)0;
        const R b11 = (vqk && vql) ? A[qk + ql * LA] : (R)0;
        // rows: [p';q'] = [c -s; s c] [p; q]
        const R r00 = ck * b00 - sk * b10, r01 = ck * b01 - sk * b11;
        const R r10 = sk * b00 + ck * b10, r11 = sk * b01 + ck * b11;
        // columns: [p' q'] = [p q] [c s; -s c]
        A[pk + pl * LA] = cl * r00 - sl * r01;
        if (vql) A[pk + ql * LA] = sl * r00 + cl * r01;
        if (vqk) A[qk + pl * LA] = cl * r10 - sl * r11;
        if (vqk && vql) A[qk + ql * LA] = sl * r10 + cl * r11;
      }
      // accumulate S <- S J
      for (int it = tid; it < j * np; it += SM_THREADS) {
        const int row = it / np, k = it % np;
        if (!rot[k]) continue;
        const int p = pp[k], q = qq[k];
        const R sp = Sm[row + p * LA], sq = Sm[row + q * LA];
        Sm[row + p * LA] = cs[k] * sp - sn[k] * sq;
        Sm[row + q * LA] = sn[k] * sp + cs[k] * sq;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    if (F64) H[r + (size_t)c * ldh] = (double)A[r + c * LA];
    S[r + (size_t)c * lds] = (double)Sm[r + c * LA];
  }
  for (int i = tid; i < j; i += SM_THREADS) theta[i] = (double)A[i + i * LA];
  if (tid == 0 && sweeps_out) sweeps_out[0] = sweep;
  if (tid == 0 && rot_out) rot_out[0] = nrot;
}

void jacobi_eig_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                   int max_sweeps, int* sweeps_out, double tol_loose, int ntarget, int tmode, double tshift,
                   int* rot_out) {
  ProfScope ps(s, PROF_JACOBI);
  const size_t smem = sizeof(double) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_jacobi_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_jacobi_eig<double><<<1, SM_THREADS, smem, s>>>(j, H, ldh, S, lds, theta, tol, max_sweeps, sweeps_out,
                                                    tol_loose, ntarget, tmode, tshift, rot_out); count_launch();
}

// ---------------------------------------------------------------------------
// The same FP64 cyclic Jacobi spread over a thread-block cluster of JC_CTAS
// CTAs (one SM's FP64 pipe is the limit of the single-CTA kernel on GB300).
// Every CTA holds a full copy of the frame matrix in its shared memory and
// computes all rotation parameters of a round itself (the copies are
// identical, so every CTA takes the same decisions); CTA c updates the 2 x 2
// blocks whose column pair l has l % JC_CTAS == c and stores the results into
// all copies through distributed shared memory; the rows of the accumulated
// rotation S are split among the CTAs.  One cluster barrier per round (a
// hardware barrier: no spin loop).
// ---------------------------------------------------------------------------
constexpr int JC_CTAS = 8;

__global__ void __cluster_dims__(JC_CTAS, 1, 1) __launch_bounds__(SM_THREADS)
    k_jacobi_eig_cluster(int j, double* H, int ldh, double* S, int lds, double* theta, double tol, int max_sweeps,
                         int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift, int* rot_out) {
  extern __shared__ __align__(16) double dsm[];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  double* A = dsm;                              // [SM_MAXJ * (SM_MAXJ + 1)]
  double* Sm = A + SM_MAXJ * (SM_MAXJ + 1);     // rows r0..r1 used
  __shared__ double cs[SM_MAXJ / 2], sn[SM_MAXJ / 2];
  __shared__ int pp[SM_MAXJ / 2], qq[SM_MAXJ / 2], rot[SM_MAXJ / 2];
  __shared__ unsigned char is_t[SM_MAXJ];
  __shared__ double scale_s;
  __shared__ double wmx[SM_THREADS / 32];
  double* Ar[JC_CTAS];
#pragma unroll
  for (int r = 0; r < JC_CTAS; ++r) Ar[r] = cl.map_shared_rank(A, r);
  const int tid = threadIdx.x;
  const int LA = SM_MAXJ + 1;
  const int rows_per = (j + JC_CTAS - 1) / JC_CTAS;
  const int r0 = crank * rows_per, r1 = min(j, r0 + rows_per);
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    A[r + c * LA] = H[r + (size_t)c * ldh];
    if (r >= r0 && r < r1) Sm[r + c * LA] = S[r + (size_t)c * lds];
  }
  __syncthreads();
  double mx = 0.0;
  for (int e = tid; e < j * j; e += SM_THREADS) mx = fmax(mx, fabs(A[(e % j) + (e / j) * LA]));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  if ((tid & 31) == 0) wmx[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int w = 0; w < SM_THREADS / 32; ++w) m2 = fmax(m2, wmx[w]);
    scale_s = m2;
  }
  cl.sync();  // every copy is loaded before any remote store
  const double thr_t = tol * scale_s;
  const double inv_scale = scale_s > 0.0 ? 1.0 / scale_s : 1.0;
  const double rel = ntarget > 0 ? tol_rel : 0.0;
  auto need = [&](int p, int q, double apq) -> bool {
    if (is_t[p] | is_t[q]) return fabs(apq) > thr_t;
    if (rel == 0.0) return fabs(apq) > thr_t;
    const float r2 = (float)rel * sqrtf(fabsf((float)(A[p + p * LA] * inv_scale) * (float)(A[q + q * LA] * inv_scale)));
    return fabs(apq) > fmax((double)r2 * scale_s, thr_t);
  };
  const int jj = j + (j & 1);
  const int np = jj / 2;
  int sweep = 0, nrot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid < j) {
      int rr = 1;
      if (ntarget > 0) {
        auto key = [&](int t2) {
          const double d = A[t2 + t2 * LA];
          return tmode == 0 ? d : (tmode == 1 ? -d : fabs(d - tshift));
        };
        const double ki = key(tid);
        int rank = 0;
        for (int t2 = 0; t2 < j; ++t2) {
          const double kt = key(t2);
          if (kt < ki || (kt == ki && t2 < tid)) ++rank;
        }
        rr = rank < ntarget;
      }
      is_t[tid] = (unsigned char)rr;
    }
    __syncthreads();
    int any = 0;
    for (int e = tid; e < j * j; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      if (r < c && need(r, c, A[r + c * LA])) any = 1;
    }
    if (!__syncthreads_or(any)) break;  // identical in every CTA
    for (int round = 0; round < jj - 1; ++round) {
      int mine = 0;
      if (tid < np) {
        int p, q;
        rr_pair(jj, round, tid, p, q);
        pp[tid] = p;
        qq[tid] = q;
        int rr = 0;
        if (q < j) {
          const double apq = A[p + q * LA];
          if (need(p, q, apq)) {
            double c, sv;
            rot_params(A[p + p * LA], A[q + q * LA], apq, inv_scale, c, sv);
            cs[tid] = c;
            sn[tid] = sv;
            rr = 1;
          }
        }
        rot[tid] = rr;
        mine = rr;
      }
      if (!__syncthreads_or(mine)) continue;  // identical in every CTA
      if (crank == 0 && tid == 0) {
        int cnt = 0;
        for (int k2 = 0; k2 < np; ++k2) cnt += rot[k2];
        nrot += cnt;
      }
      // this CTA's column pairs: l = crank, crank + JC_CTAS, ...; four threads
      // per 2 x 2 block (k, l), one per output element (a, c): a thread issues
      // 6 FP64 instructions instead of a whole block's 16, and 8 remote stores
      // instead of 32 (one FP64 warp instruction holds a sub-partition's FP64
      // pipe for many cycles on GB300, so instructions per warp set the time)
      const int nl = (np - crank + JC_CTAS - 1) / JC_CTAS;
      const int nitems = np * nl * 4;
      // warp-uniform trip count: the four threads of a block are lanes of one
      // warp, and every lane reads its block's inputs before any lane writes
      // (__syncwarp between the two)
      for (int it0 = tid & ~31; it0 < nitems; it0 += SM_THREADS) {
        const int it = it0 + (tid & 31);
        const int blk = it >> 2, ea = (it >> 1) & 1, ec = it & 1;
        const int k = blk % np, l = crank + (blk / np) * JC_CTAS;
        bool upd = false, diag = false;
        int pk = 0, qk = 0, pl = 0, ql = 0;
        double out = 0.0, n00 = 0.0, n11 = 0.0, n01 = 0.0;
        if (it < nitems && (rot[k] || rot[l])) {
          pk = pp[k];
          qk = qq[k];
          pl = pp[l];
          ql = qq[l];
          const bool vqk = qk < j, vql = ql < j;
          if (k == l) {
            if (vqk && ea == 0 && ec == 0) {  // full 2 x 2 update J^T B J (the angle is not exact)
              const double c = cs[k], sv = sn[k];
              const double app = A[pk + pk * LA], aqq = A[qk + qk * LA], apq = A[pk + qk * LA];
              const double r00 = c * app - sv * apq, r01 = c * apq - sv * aqq;
              const double r10 = sv * app + c * apq, r11 = sv * apq + c * aqq;
              n00 = c * r00 - sv * r01;
              n11 = sv * r10 + c * r11;
              n01 = (sv * r00 + c * r01 + c * r10 - sv * r11) * 0.5;
              diag = true;
            }
          } else if (!((ea && !vqk) || (ec && !vql))) {  // skip outputs outside the matrix (odd j)
            const int rk = rot[k], rl = rot[l];
            const double ck = rk ? cs[k] : 1.0, sk = rk ? sn[k] : 0.0;
            const double cl2 = rl ? cs[l] : 1.0, sl = rl ? sn[l] : 0.0;
            const double b00 = A[pk + pl * LA];
            const double b01 = vql ? A[pk + ql * LA] : 0.0;
            const double b10 = vqk ? A[qk + pl * LA] : 0.0;
            const double b11 = (vqk && vql) ? A[qk + ql * LA] : 0.0;
            // rows: [p'; q'] = [c -s; s c] [p; q]; columns: [p' q'] = [p q] [c s; -s c]
            const double ra0 = ea ? sk * b00 + ck * b10 : ck * b00 - sk * b10;
            const double ra1 = ea ? sk * b01 + ck * b11 : ck * b01 - sk * b11;
            out = ec ? sl * ra0 + cl2 * ra1 : cl2 * ra0 - sl * ra1;
            upd = true;
          }
        }
        __syncwarp();
        if (diag) {
#pragma unroll
          for (int r = 0; r < JC_CTAS; ++r) {
            Ar[r][pk + pk * LA] = n00;
            Ar[r][qk + qk * LA] = n11;
            Ar[r][pk + qk * LA] = n01;
            Ar[r][qk + pk * LA] = n01;
          }
        } else if (upd) {
          const int ri = ea ? qk : pk, cj = ec ? ql : pl;
#pragma unroll
          for (int r = 0; r < JC_CTAS; ++r) Ar[r][ri + cj * LA] = out;
        }
      }
      // the rows of S this CTA owns
      for (int it = tid; it < (r1 - r0) * np; it += SM_THREADS) {
        const int row = r0 + it / np, k = it % np;
        if (!rot[k]) continue;
        const int p = pp[k], q = qq[k];
        const double sp = Sm[row + p * LA], sq = Sm[row + q * LA];
        Sm[row + p * LA] = cs[k] * sp - sn[k] * sq;
        Sm[row + q * LA] = sn[k] * sp + cs[k] * sq;
      }
      cl.sync();
    }
  }
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    if (crank == 0) H[r + (size_t)c * ldh] = A[r + c * LA];
    if (r >= r0 && r < r1) S[r + (size_t)c * lds] = Sm[r + c * LA];
  }
  if (crank == 0) {
    for (int i = tid; i < j; i += SM_THREADS) theta[i] = A[i + i * LA];
    if (tid == 0 && sweeps_out) sweeps_out[0] = sweep;
    if (tid == 0 && rot_out) rot_out[0] = nrot;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

void jacobi_eig_cluster_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                           int max_sweeps, int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift,
                           int* rot_out) {
  ProfScope ps(s, PROF_JACOBI);
  const size_t smem = sizeof(double) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_jacobi_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_jacobi_eig_cluster<<<JC_CTAS, SM_THREADS, smem, s>>>(j, H, ldh, S, lds, theta, tol, max_sweeps, sweeps_out,
                                                          tol_rel, ntarget, tmode, tshift, rot_out); count_launch();
}

void jacobi_eig32_ld(cudaStream_t s, int j, const double* H, int ldh, double* Sf, int lds, double* theta, double tol,
                     int max_sweeps, int* sweeps_out, int* rot_out) {
  ProfScope ps(s, PROF_JACOBI);
  const size_t smem = sizeof(float) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  k_jacobi_eig<float><<<1, SM_THREADS, smem, s>>>(j, const_cast<double*>(H), ldh, Sf, lds, theta, tol, max_sweeps,
                                                   sweeps_out, tol, 0, 0, 0.0, rot_out); count_launch();
}
// ---------------------------------------------------------------------------
// The same two-sided Jacobi (same pairing, thresholds, targets and update
// formulas) in one CTA with each round's work compacted:
//  * the rotation parameters of the round's pairs are spread over 4 warps
//    (one per SM sub-partition): pair k is lane k/4 of warp k%4;
//  * only the 2 x 2 blocks (k, l) with a rotating pair are updated, the
//    upper triangle of them (k rotating; (l, k) written as the transpose),
//    packed densely into as few warps as possible;
//  * S is updated for the rotating pairs only;
//  * a round has two CTA barriers and no cluster barrier.
// Measured on GB300 it is no faster than the 8-CTA cluster kernel (about
// 0.6 ms against 0.55 ms per stage-1 call at j ~ 27): a round is bound by
// the serial chain of its rotation parameters and barriers, not by the
// update flops, so it is the kernel-level one-CTA entry point and an option
// of the solver, not its default.
// Pair k has the bit position (k % 4) * 8 + k / 4 in the round's mask M.
// ---------------------------------------------------------------------------
__device__ inline int jf_pair_of_bit(int b) { return (b & 7) * 4 + (b >> 3); }
__device__ inline int jf_bit_of_pair(int k) { return (k & 3) * 8 + (k >> 2); }

__global__ void __launch_bounds__(SM_THREADS)
    k_jacobi_eig_fast(int j, double* H, int ldh, double* S, int lds, double* theta, double tol, int max_sweeps,
                      int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift, int* rot_out) {
  extern __shared__ __align__(16) double dsm[];
  double* A = dsm;                              // [SM_MAXJ * (SM_MAXJ + 1)]
  double* Sm = A + SM_MAXJ * (SM_MAXJ + 1);
  __shared__ double cs[SM_MAXJ / 2], sn[SM_MAXJ / 2];
  __shared__ int pp[SM_MAXJ / 2], qq[SM_MAXJ / 2];
  __shared__ unsigned pmask[2][4];  // by round parity: a round without rotations skips the closing barrier
  __shared__ unsigned char is_t[SM_MAXJ];
  __shared__ double scale_s;
  __shared__ double wmx[SM_THREADS / 32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int LA = SM_MAXJ + 1;
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    A[r + c * LA] = H[r + (size_t)c * ldh];
    Sm[r + c * LA] = S[r + (size_t)c * lds];
  }
  __syncthreads();
  double mx = 0.0;
  for (int e = tid; e < j * j; e += SM_THREADS) mx = fmax(mx, fabs(A[(e % j) + (e / j) * LA]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) wmx[w] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int k = 0; k < SM_THREADS / 32; ++k) m2 = fmax(m2, wmx[k]);
    scale_s = m2;
  }
  __syncthreads();
  const double thr_t = tol * scale_s;
  const double inv_scale = scale_s > 0.0 ? 1.0 / scale_s : 1.0;
  const double rel = ntarget > 0 ? tol_rel : 0.0;
  auto need = [&](int p, int q, double apq) -> bool {
    if (is_t[p] | is_t[q]) return fabs(apq) > thr_t;
    if (rel == 0.0) return fabs(apq) > thr_t;
    const float r2 =
        (float)rel * sqrtf(fabsf((float)(A[p + p * LA] * inv_scale) * (float)(A[q + q * LA] * inv_scale)));
    return fabs(apq) > fmax((double)r2 * scale_s, thr_t);
  };
  const int jj = j + (j & 1);
  const int np = jj / 2;
  int sweep = 0, nrot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid < j) {
      int rr = 1;
      if (ntarget > 0) {
        auto key = [&](int t2) {
          const double d = A[t2 + t2 * LA];
          return tmode == 0 ? d : (tmode == 1 ? -d : fabs(d - tshift));
        };
        const double ki = key(tid);
        int rank = 0;
        for (int t2 = 0; t2 < j; ++t2) {
          const double kt = key(t2);
          if (kt < ki || (kt == ki && t2 < tid)) ++rank;
        }
        rr = rank < ntarget;
      }
      is_t[tid] = (unsigned char)rr;
    }
    __syncthreads();
    int any = 0;
    for (int e = tid; e < j * j; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      if (r < c && need(r, c, A[r + c * LA])) any = 1;
    }
    if (!__syncthreads_or(any)) break;
    for (int round = 0; round < jj - 1; ++round) {
      bool mine = false;
      if (w < 4 && lane < 8) {
        const int k = lane * 4 + w;
        if (k < np) {
          int p, q;
          rr_pair(jj, round, k, p, q);
          pp[k] = p;
          qq[k] = q;
          if (q < j) {
            const double apq = A[p + q * LA];
            if (need(p, q, apq)) {
              double c, sv;
              rot_params(A[p + p * LA], A[q + q * LA], apq, inv_scale, c, sv);
              cs[k] = c;
              sn[k] = sv;
              mine = true;
            }
          }
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      unsigned* pm = pmask[round & 1];
      if (w < 4 && lane == 0) pm[w] = bal & 0xffu;
      __syncthreads();
      const unsigned M = pm[0] | (pm[1] << 8) | (pm[2] << 16) | (pm[3] << 24);
      if (M == 0) continue;  // the same M in every thread
      const int nr = __popc(M);
      if (tid == 0) nrot += nr;
      // 2 x 2 blocks (k, l), k rotating: rows of pair k, columns of pair l
      for (int it = tid; it < nr * np; it += SM_THREADS) {
        const int a = it / np, l = it % np;
        const int k = jf_pair_of_bit(__fns(M, 0, a + 1));
        const int bl = jf_bit_of_pair(l);
        const bool rl = (M >> bl) & 1u;
        if (rl && __popc(M & ((1u << bl) - 1u)) < a) continue;  // (l, k) is the transpose of a done block
        const int pk = pp[k], qk = qq[k], pl = pp[l], ql = qq[l];
        const double ck = cs[k], sk = sn[k];
        if (l == k) {  // full 2 x 2 update J^T B J (the angle is not exact)
          const double app = A[pk + pk * LA], aqq = A[qk + qk * LA], apq = A[pk + qk * LA];
          const double r00 = ck * app - sk * apq, r01 = ck * apq - sk * aqq;
          const double r10 = sk * app + ck * apq, r11 = sk * apq + ck * aqq;
          const double n00 = ck * r00 - sk * r01, n11 = sk * r10 + ck * r11;
          const double n01 = (sk * r00 + ck * r01 + ck * r10 - sk * r11) * 0.5;
          A[pk + pk * LA] = n00;
          A[qk + qk * LA] = n11;
          A[pk + qk * LA] = n01;
          A[qk + pk * LA] = n01;
          continue;
        }
        const double cl2 = rl ? cs[l] : 1.0, sl = rl ? sn[l] : 0.0;
        const bool vql = ql < j;
        const double b00 = A[pk + pl * LA];
        const double b01 = vql ? A[pk + ql * LA] : 0.0;
        const double b10 = A[qk + pl * LA];
        const double b11 = vql ? A[qk + ql * LA] : 0.0;
        const double r00 = ck * b00 - sk * b10, r01 = ck * b01 - sk * b11;
        const double r10 = sk * b00 + ck * b10, r11 = sk * b01 + ck * b11;
        const double n00 = cl2 * r00 - sl * r01, n01 = sl * r00 + cl2 * r01;
        const double n10 = cl2 * r10 - sl * r11, n11 = sl * r10 + cl2 * r11;
        A[pk + pl * LA] = n00;
        A[qk + pl * LA] = n10;
        A[pl + pk * LA] = n00;
        A[pl + qk * LA] = n10;
        if (vql) {
          A[pk + ql * LA] = n01;
          A[qk + ql * LA] = n11;
          A[ql + pk * LA] = n01;
          A[ql + qk * LA] = n11;
        }
      }
      // S <- S J on the columns of the rotating pairs (packed from warp 7 down,
      // so they share the sub-partitions with the fewest block updates)
      for (int it = SM_THREADS - 1 - tid; it < nr * j; it += SM_THREADS) {
        const int a = it / j, row = it % j;
        const int k = jf_pair_of_bit(__fns(M, 0, a + 1));
        const int p = pp[k], q = qq[k];
        const double sp = Sm[row + p * LA], sq = Sm[row + q * LA];
        Sm[row + p * LA] = cs[k] * sp - sn[k] * sq;
        Sm[row + q * LA] = sn[k] * sp + cs[k] * sq;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    H[r + (size_t)c * ldh] = A[r + c * LA];
    S[r + (size_t)c * lds] = Sm[r + c * LA];
  }
  for (int i = tid; i < j; i += SM_THREADS) theta[i] = A[i + i * LA];
  if (tid == 0 && sweeps_out) sweeps_out[0] = sweep;
  if (tid == 0 && rot_out) rot_out[0] = nrot;
}

// ---------------------------------------------------------------------------
// FP64 clean-up of the target pairs after an FP32 Jacobi pass: only pairs that
// touch one of the ntarget targets (smallest diagonal entries for tmode 0,
// largest for 1, closest to tshift for 2, ranked once per sweep) are rotated,
// to the absolute threshold tol * max|a_ij|; pairs between two non-targets are
// left as the FP32 pass made them.  A sweep is (a) nN rounds in which target i
// pairs with non-target N[(r + i) mod nN] (disjoint, nt <= nN) and (b) the
// round-robin rounds of the target-target pairs.  Each round: rotation
// parameters of its <= 8 pairs in one warp, then the row rotations (and S's
// columns), then the column rotations -- two-sided J^T A J with disjoint
// pairs.  After the FP32 pass the angles are small: for |t| < 2^-10 the
// cosine is the series 1 - t^2/2 + 3 t^4/8 (error below 2^-60) instead of
// the rsqrt refinement, which shortens the serial FP64 chain of a round.
// ---------------------------------------------------------------------------
constexpr int JT_MAXT = 8;

__device__ inline void rot_params_small(double app, double aqq, double apq, double inv_scale, double& c, double& s_) {
  const float fpp = (float)(app * inv_scale), fqq = (float)(aqq * inv_scale), fpq = (float)(apq * inv_scale);
  const float ftau = (fqq - fpp) / (2.0f * fpq);
  const float ft = copysignf(1.0f, ftau) / (fabsf(ftau) + sqrtf(1.0f + ftau * ftau));
  if (fabsf(ft) < 0.0009765625f) {
    const double t = (double)ft;
    const double t2 = t * t;
    const double cc = fma(t2, fma(t2, 0.375, -0.5), 1.0);
    c = cc;
    s_ = t * cc;
  } else {
    rot_params(app, aqq, apq, inv_scale, c, s_);
  }
}

__global__ void __launch_bounds__(SM_THREADS)
    k_jacobi_targets(int j, double* H, int ldh, double* S, int lds, double* theta, double tol, int max_sweeps,
                     int* sweeps_out, int ntarget, int tmode, double tshift, int* rot_out) {
  extern __shared__ __align__(16) double dsm[];
  double* A = dsm;                              // [SM_MAXJ * (SM_MAXJ + 1)]
  double* Sm = A + SM_MAXJ * (SM_MAXJ + 1);
  __shared__ double cs[JT_MAXT], sn[JT_MAXT];
  __shared__ int pp[JT_MAXT], qq[JT_MAXT], rotf[JT_MAXT];
  __shared__ int tgt[JT_MAXT], non[SM_MAXJ];
  __shared__ int nt_s, nn_s;
  __shared__ double scale_s;
  __shared__ double wmx[SM_THREADS / 32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int LA = SM_MAXJ + 1;
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    A[r + c * LA] = H[r + (size_t)c * ldh];
    Sm[r + c * LA] = S[r + (size_t)c * lds];
  }
  __syncthreads();
  double mx = 0.0;
  for (int e = tid; e < j * j; e += SM_THREADS) mx = fmax(mx, fabs(A[(e % j) + (e / j) * LA]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) wmx[w] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int k = 0; k < SM_THREADS / 32; ++k) m2 = fmax(m2, wmx[k]);
    scale_s = m2;
  }
  __syncthreads();
  const double thr = tol * scale_s;
  const double inv_scale = scale_s > 0.0 ? 1.0 / scale_s : 1.0;
  int sweep = 0, nrot = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // rank the targets on the current diagonal
    if (tid == 0) {
      nt_s = 0;
      nn_s = 0;
    }
    __syncthreads();
    if (tid < j) {
      auto key = [&](int t2) {
        const double d = A[t2 + t2 * LA];
        const double k = tmode == 0 ? d : (tmode == 1 ? -d : fabs(d - tshift));
        return isnan(k) ? INFINITY : k;
      };
      const double ki = key(tid);
      int rank = 0;
      for (int t2 = 0; t2 < j; ++t2) {
        const double kt = key(t2);
        if (kt < ki || (kt == ki && t2 < tid)) ++rank;
      }
      const int ntg = ntarget < JT_MAXT ? ntarget : JT_MAXT;
      if (rank < ntg && rank < j - 1) tgt[rank] = tid;
    }
    __syncthreads();
    if (tid == 0) {
      const int ntg = min(min(ntarget, JT_MAXT), j - 1);
      nt_s = ntg > 0 ? ntg : 0;
      int c = 0;
      for (int i = 0; i < j; ++i) {
        bool is_t = false;
        for (int a = 0; a < nt_s; ++a) is_t |= tgt[a] == i;
        if (!is_t) non[c++] = i;
      }
      nn_s = c;
    }
    __syncthreads();
    const int nt = nt_s, nn = nn_s;
    // converged: every pair touching a target below the threshold
    int any = 0;
    for (int e = tid; e < nt * j; e += SM_THREADS) {
      const int a = e / j, x = e % j, t = tgt[a];
      if (x != t && fabs(A[t + x * LA]) > thr) any = 1;
    }
    if (!__syncthreads_or(any)) break;
    // (a) every target-non-target pair once: max(nt, nn) rounds of disjoint
    // pairs (the smaller side by lane, the larger one shifted each round)
    // (b) the target-target pairs, round robin
    const int ntt = nt + (nt & 1);
    const int na = nt > 0 ? (nt > nn ? nt : nn) : 0;
    const int nrounds = na + (nt > 1 ? ntt - 1 : 0);
    for (int round = 0; round < nrounds; ++round) {
      bool mine = false;
      if (w == 0 && lane < JT_MAXT) {
        int p = -1, q = -1;
        if (round < na) {
          if (nt <= nn) {
            if (lane < nt) {
              p = tgt[lane];
              q = non[(round + lane) % nn];
            }
          } else if (lane < nn) {
            p = tgt[(round + lane) % nt];
            q = non[lane];
          }
        } else if (lane < ntt / 2) {
          int a, b;
          rr_pair(ntt, round - na, lane, a, b);
          if (b < nt) {
            p = tgt[a];
            q = tgt[b];
          }
        }
        rotf[lane] = 0;
        if (p >= 0) {
          if (p > q) {
            const int tmp = p;
            p = q;
            q = tmp;
          }
          pp[lane] = p;
          qq[lane] = q;
          const double apq = A[p + q * LA];
          if (fabs(apq) > thr) {
            double c, sv;
            rot_params_small(A[p + p * LA], A[q + q * LA], apq, inv_scale, c, sv);
            cs[lane] = c;
            sn[lane] = sv;
            rotf[lane] = 1;
            mine = true;
          }
        }
      }
      if (!__syncthreads_or(mine)) continue;
      if (tid == 0)
        for (int k = 0; k < JT_MAXT; ++k) nrot += rotf[k];
      // rows p, q of A and columns p, q of S
      for (int it = tid; it < JT_MAXT * j; it += SM_THREADS) {
        const int k = it / j, x = it % j;
        if (!rotf[k]) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], sv = sn[k];
        const double ap = A[p + x * LA], aq = A[q + x * LA];
        A[p + x * LA] = c * ap - sv * aq;
        A[q + x * LA] = sv * ap + c * aq;
        const double sp = Sm[x + p * LA], sq = Sm[x + q * LA];
        Sm[x + p * LA] = c * sp - sv * sq;
        Sm[x + q * LA] = sv * sp + c * sq;
      }
      __syncthreads();
      // columns p, q of A
      for (int it = tid; it < JT_MAXT * j; it += SM_THREADS) {
        const int k = it / j, x = it % j;
        if (!rotf[k]) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], sv = sn[k];
        const double ap = A[x + p * LA], aq = A[x + q * LA];
        A[x + p * LA] = c * ap - sv * aq;
        A[x + q * LA] = sv * ap + c * aq;
      }
      __syncthreads();
      // keep each rotated 2 x 2 diagonal block exactly symmetric
      if (tid < JT_MAXT && rotf[tid]) {
        const int p = pp[tid], q = qq[tid];
        const double v = 0.5 * (A[p + q * LA] + A[q + p * LA]);
        A[p + q * LA] = v;
        A[q + p * LA] = v;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    H[r + (size_t)c * ldh] = A[r + c * LA];
    S[r + (size_t)c * lds] = Sm[r + c * LA];
  }
  for (int i = tid; i < j; i += SM_THREADS) theta[i] = A[i + i * LA];
  if (tid == 0 && sweeps_out) sweeps_out[0] = sweep;
  if (tid == 0 && rot_out) rot_out[0] = nrot;
}

void jacobi_eig_targets_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                           int max_sweeps, int* sweeps_out, int ntarget, int tmode, double tshift, int* rot_out) {
  ProfScope ps(s, PROF_JACOBI);
  const size_t smem = sizeof(double) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_jacobi_targets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_jacobi_targets<<<1, SM_THREADS, smem, s>>>(j, H, ldh, S, lds, theta, tol, max_sweeps, sweeps_out, ntarget,
                                               tmode, tshift, rot_out);
  count_launch();
}

void jacobi_eig_fast_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                        int max_sweeps, int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift,
                        int* rot_out) {
  ProfScope ps(s, PROF_JACOBI);
  const size_t smem = sizeof(double) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_jacobi_eig_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_jacobi_eig_fast<<<1, SM_THREADS, smem, s>>>(j, H, ldh, S, lds, theta, tol, max_sweeps, sweeps_out, tol_rel,
                                                ntarget, tmode, tshift, rot_out);
  count_launch();
}

void jacobi_eig(cudaStream_t s, int j, double* H, double* S, double* theta, double tol, int max_sweeps,
                int* sweeps_out) {
  jacobi_eig_ld(s, j, H, j, S, j, theta, tol, max_sweeps, sweeps_out, tol, 0, 0, 0.0, nullptr);
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD: rotate column pairs of G until
// |g_p^T g_q| <= tol * ||g_p|| ||g_q|| for all pairs (relative accuracy).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SM_THREADS) k_jacobi_svd(int j, double* G, int ldg, double* S, int lds,
                                                           double* sig, double tol, int max_sweeps,
                                                           int* sweeps_out) {
  extern __shared__ __align__(16) double dsm[];
  double* Gm = dsm;                             // [SM_MAXJ * (SM_MAXJ + 1)]
  double* Sm = Gm + SM_MAXJ * (SM_MAXJ + 1);    // [SM_MAXJ * (SM_MAXJ + 1)]
  __shared__ double cs[SM_MAXJ / 2], sn[SM_MAXJ / 2];
  __shared__ int pp[SM_MAXJ / 2], qq[SM_MAXJ / 2], rot[SM_MAXJ / 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int LA = SM_MAXJ + 1;
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    Gm[r + c * LA] = G[r + (size_t)c * ldg];
    Sm[r + c * LA] = S[r + (size_t)c * lds];
  }
  __syncthreads();
  const int jj = j + (j & 1);
  const int np = jj / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int any_sweep = 0;
    for (int round = 0; round < jj - 1; ++round) {
      // one warp per pair: the three inner products
      for (int k = warp; k < np; k += SM_THREADS / 32) {
        int p, q;
        rr_pair(jj, round, k, p, q);
        double a = 0.0, b = 0.0, g = 0.0;
        if (q < j) {
          for (int r = lane; r < j; r += 32) {
            const double gp = Gm[r + p * LA], gq = Gm[r + q * LA];
            a = fma(gp, gp, a);
            b = fma(gq, gq, b);
            g = fma(gp, gq, g);
          }
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (lane == 0) {
          pp[k] = p;
          qq[k] = q;
          int r = 0;
          if (q < j && g != 0.0 && fabs(g) > tol * sqrt(a * b)) {
            const double zeta = (b - a) / (2.0 * g);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            cs[k] = c;
            sn[k] = c * t;
            r = 1;
          }
          rot[k] = r;
        }
      }
      __syncthreads();
      int mine = 0;
      if (tid < np) mine = rot[tid];
      if (!__syncthreads_or(mine)) continue;
      any_sweep = 1;
      for (int it = tid; it < j * np; it += SM_THREADS) {
        const int row = it / np, k = it % np;
        if (!rot[k]) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s_ = sn[k];
        const double gp = Gm[row + p * LA], gq = Gm[row + q * LA];
        Gm[row + p * LA] = c * gp - s_ * gq;
        Gm[row + q * LA] = s_ * gp + c * gq;
        const double sp = Sm[row + p * LA], sq = Sm[row + q * LA];
        Sm[row + p * LA] = c * sp - s_ * sq;
        Sm[row + q * LA] = s_ * sp + c * sq;
      }
      __syncthreads();
    }
    if (!any_sweep) break;
  }
  for (int e = tid; e < j * j; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    G[r + (size_t)c * ldg] = Gm[r + c * LA];
    S[r + (size_t)c * lds] = Sm[r + c * LA];
  }
  __syncthreads();
  for (int c = warp; c < j; c += SM_THREADS / 32) {
    double a = 0.0;
    for (int r = lane; r < j; r += 32) a = fma(Gm[r + c * LA], Gm[r + c * LA], a);
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrt(a);
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

void jacobi_svd_ld(cudaStream_t s, int j, double* G, int ldg, double* S, int lds, double* sig, double tol,
                   int max_sweeps, int* sweeps_out) {
  ProfScope ps(s, PROF_SMALL);
  const size_t smem = sizeof(double) * 2 * SM_MAXJ * (SM_MAXJ + 1);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_jacobi_svd<<<1, SM_THREADS, smem, s>>>(j, G, ldg, S, lds, sig, tol, max_sweeps, sweeps_out); count_launch();
}
void jacobi_svd(cudaStream_t s, int j, double* G, double* S, double* sig, double tol, int max_sweeps,
                int* sweeps_out) {
  jacobi_svd_ld(s, j, G, j, S, j, sig, tol, max_sweeps, sweeps_out);
}

// ---------------------------------------------------------------------------
// Cholesky of the q x q Gram P = L L^T (q <= 8), M = L^{-T} (upper triangular),
// flags[c] = 1 when pivot^2 < drop^2 * in_norm2[c]: column c of the block is
// numerically in the span of the basis and the previous block columns.
// ---------------------------------------------------------------------------
__global__ void k_chol(int q, const double* __restrict__ P, const double* __restrict__ in_norm2, double drop,
                       double* __restrict__ M, int* __restrict__ flags) {
  if (threadIdx.x != 0) return;
  double L[8][8];
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) L[a][b] = 0.0;
  int bad = 0;
  for (int c = 0; c < q; ++c) {
    double d = P[c + c * q];
    for (int k = 0; k < c; ++k) d -= L[c][k] * L[c][k];
    const double ref = in_norm2 ? in_norm2[c] : P[c + c * q];
    int f = 0;
    if (!(d > drop * drop * ref) || !(d > 0.0)) {
      f = 1;
      d = 1.0;  // keep the factor finite; the caller replaces the column
    }
    flags[c] = f;
    bad |= f;
    const double lcc = sqrt(d);
    L[c][c] = lcc;
    for (int r = c + 1; r < q; ++r) {
      double v = P[r + c * q];
      for (int k = 0; k < c; ++k) v -= L[r][k] * L[c][k];
      L[r][c] = f ? 0.0 : v / lcc;
    }
  }
  // M = L^{-T}: solve L^T M = I (upper triangular M)
  for (int c = 0; c < q; ++c) {
    for (int r = q - 1; r >= 0; --r) {
      double v = (r == c) ? 1.0 : 0.0;
      for (int k = r + 1; k < q; ++k) v -= L[k][r] * M[k + c * q];
      M[r + c * q] = v / L[r][r];
    }
  }
  flags[q] = bad;
}
void chol_factor(cudaStream_t s, int q, const double* P, const double* in_norm2, double drop, double* M,
                 int* flags) {
  k_chol<<<1, 32, 0, s>>>(q, P, in_norm2, drop, M, flags); count_launch();
}

// ---------------------------------------------------------------------------
// Small dense products on several CTAs (one thread per output entry).
// ---------------------------------------------------------------------------
__global__ void k_gemm_tn(int a, int r, int c, const double* __restrict__ A, int lda, const double* __restrict__ B,
                          int ldb, double* __restrict__ C, int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  const int i = e % r, k = e / r;
  double acc = 0.0;
  for (int t = 0; t < a; ++t) acc = fma(A[t + (size_t)i * lda], B[t + (size_t)k * ldb], acc);
  C[i + (size_t)k * ldc] = acc;
}
__global__ void k_gemm_nn(int r, int a, int c, const double* __restrict__ A, int lda, const double* __restrict__ B,
                          int ldb, double* __restrict__ C, int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  const int i = e % r, k = e / r;
  double acc = 0.0;
  for (int t = 0; t < a; ++t) acc = fma(A[i + (size_t)t * lda], B[t + (size_t)k * ldb], acc);
  C[i + (size_t)k * ldc] = acc;
}
void small_gemm_tn(cudaStream_t s, int a, int r, int c, const double* A, int lda, const double* B, int ldb,
                   double* C, int ldc) {
  if (r * c > 0) k_gemm_tn<<<ceil_div(r * c, 64), 64, 0, s>>>(a, r, c, A, lda, B, ldb, C, ldc); count_launch();
}
void small_gemm_nn(cudaStream_t s, int r, int a, int c, const double* A, int lda, const double* B, int ldb,
                   double* C, int ldc) {
  if (r * c > 0) k_gemm_nn<<<ceil_div(r * c, 64), 64, 0, s>>>(r, a, c, A, lda, B, ldb, C, ldc); count_launch();
}

// ---------------------------------------------------------------------------
// Append nb new basis vectors to the Jacobi frame.  Hnew ((j0+nb) x nb, ld
// j0+nb) holds V^T W_new in basis coordinates.  A (frame matrix) gets
// A[0:j0, j0+c] = S[:, 0:j0]^T Hnew[0:j0, c], A[j0+a, j0+c] = sym(Hnew[j0+a, c])
// and the mirrored lower part; S becomes blockdiag(S, I).
// ---------------------------------------------------------------------------
__global__ void k_frame_append(int j0, int nb, double* A, int lda, double* S, int lds, const double* __restrict__ Hn) {
  const int tid = threadIdx.x;
  const int ldh = j0 + nb;
  for (int e = tid; e < j0 * nb; e += blockDim.x) {
    const int i = e % j0, c = e / j0;
    double acc = 0.0;
    for (int r = 0; r < j0; ++r) acc = fma(S[r + (size_t)i * lds], Hn[r + (size_t)c * ldh], acc);
    A[i + (size_t)(j0 + c) * lda] = acc;
    A[(j0 + c) + (size_t)i * lda] = acc;
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int a = e % nb, c = e / nb;
    const double v = 0.5 * (Hn[(j0 + a) + (size_t)c * ldh] + Hn[(j0 + c) + (size_t)a * ldh]);
    A[(j0 + a) + (size_t)(j0 + c) * lda] = v;
  }
  const int jn = j0 + nb;
  for (int e = tid; e < jn * nb; e += blockDim.x) {
    const int r = e % jn, c = e / jn;
    S[r + (size_t)(j0 + c) * lds] = (r == j0 + c) ? 1.0 : 0.0;  // new columns
    if (r < j0) S[(j0 + c) + (size_t)r * lds] = 0.0;            // new rows of old columns
  }
}
void frame_append(cudaStream_t s, int j0, int nb, double* A, int lda, double* S, int lds, const double* Hn) {
  k_frame_append<<<1, SM_THREADS, 0, s>>>(j0, nb, A, lda, S, lds, Hn); count_launch();
}

// Append nb new basis vectors to the projected matrix H (basis coordinates):
// H[0:j0+nb, j0+c] = Hn[:, c] with the new diagonal block symmetrised and the
// mirrored rows; the rotation S becomes blockdiag(S, I).
__global__ void k_h_append(int j0, int nb, double* H, int ldh, double* S, int lds, const double* __restrict__ Hn) {
  const int jn = j0 + nb;
  for (int e = threadIdx.x; e < jn * nb; e += blockDim.x) {
    const int r = e % jn, c = e / jn;
    double v = Hn[r + (size_t)c * jn];
    if (r >= j0) v = 0.5 * (v + Hn[(j0 + c) + (size_t)(r - j0) * jn]);
    H[r + (size_t)(j0 + c) * ldh] = v;
    H[(j0 + c) + (size_t)r * ldh] = v;
    S[r + (size_t)(j0 + c) * lds] = (r == j0 + c) ? 1.0 : 0.0;
    if (r < j0) S[(j0 + c) + (size_t)r * lds] = 0.0;
  }
}
void h_append(cudaStream_t s, int j0, int nb, double* H, int ldh, double* S, int lds, const double* Hn) {
  k_h_append<<<1, SM_THREADS, 0, s>>>(j0, nb, H, ldh, S, lds, Hn); count_launch();
}

// F <- 1.5 I - 0.5 F (one Newton-Schulz step for the orthonormal polar factor:
// S <- S (3I - S^T S) / 2).
__global__ void k_ns_factor(int j, double* F, int ldf) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < j * j; e += blockDim.x * gridDim.x) {
    const int r = e % j, c = e / j;
    F[r + (size_t)c * ldf] = (r == c ? 1.5 : 0.0) - 0.5 * F[r + (size_t)c * ldf];
  }
}
void ns_factor(cudaStream_t s, int j, double* F, int ldf) { k_ns_factor<<<ceil_div(j * j, 256), 256, 0, s>>>(j, F, ldf); count_launch(); }

// A <- (A + A^T) / 2
__global__ void k_symmetrise(int j, double* A, int lda) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < j * j; e += blockDim.x * gridDim.x) {
    const int r = e % j, c = e / j;
    if (r < c) {
      const double v = 0.5 * (A[r + (size_t)c * lda] + A[c + (size_t)r * lda]);
      A[r + (size_t)c * lda] = v;
      A[c + (size_t)r * lda] = v;
    }
  }
}
void symmetrise(cudaStream_t s, int j, double* A, int lda) {
  k_symmetrise<<<ceil_div(j * j, 256), 256, 0, s>>>(j, A, lda); count_launch();
}

// Sort order of theta (j <= 64): mode 0 ascending, 1 descending, 2 ascending |theta - shift|.
// A NaN key ranks last (as +inf, ties by index), so order is always a
// permutation of 0..j-1 even when the values are not finite: the gathers that
// read it never see an unwritten slot (the host rejects the NaN afterwards).
__global__ void k_order(int j, const double* __restrict__ th, int mode, double shift, int* __restrict__ order) {
  const int i = threadIdx.x;
  if (i >= j) return;
  // mode 3 (the positive eigenvalues of B nearest zero): ascending among the
  // values above 1e-12 of the largest magnitude, the others after them
  double big = 0.0;
  if (mode == 3)
    for (int t = 0; t < j; ++t) big = fmax(big, fabs(th[t]));
  auto key = [&](int t) {
    const double k = mode == 0 ? th[t]
                   : mode == 1 ? -th[t]
                   : mode == 2 ? fabs(th[t] - shift)
                               : (th[t] > 1e-12 * big ? th[t] : INFINITY);
    return isnan(k) ? INFINITY : k;
  };
  const double ki = key(i);
  int rank = 0;
  for (int t = 0; t < j; ++t) {
    const double kt = key(t);
    if (kt < ki || (kt == ki && t < i)) ++rank;
  }
  order[rank] = i;
}
void order_theta(cudaStream_t s, int j, const double* th, int mode, double shift, int* order) {
  k_order<<<1, SM_MAXJ, 0, s>>>(j, th, mode, shift, order); count_launch();
}

// out[:, c] = S[:, idx[c]] (j rows), th_out[c] = th[idx[c]].  An index
// outside [0, j) (a corrupted ordering) is not followed: column 0 is read
// instead and *bad (when given) is set, for the host to reject the step.
__global__ void k_gather(int j, const double* __restrict__ S, int lds, const int* __restrict__ idx, int nc,
                         double* __restrict__ out, int ldo, const double* __restrict__ th, double* __restrict__ th_out,
                         int* __restrict__ bad) {
  for (int e = threadIdx.x; e < j * nc; e += blockDim.x) {
    const int r = e % j, c = e / j;
    int ic = idx[c];
    if ((unsigned)ic >= (unsigned)j) {
      if (bad) *bad = 1;
      ic = 0;
    }
    out[r + (size_t)c * ldo] = S[r + (size_t)ic * lds];
  }
  if (th && threadIdx.x < nc) {
    const int ic = idx[threadIdx.x];
    th_out[threadIdx.x] = th[(unsigned)ic < (unsigned)j ? ic : 0];
  }
}
void gather_cols(cudaStream_t s, int j, const double* S, int lds, const int* idx, int nc, double* out, int ldo,
                 const double* th, double* th_out, int* bad) {
  k_gather<<<1, SM_THREADS, 0, s>>>(j, S, lds, idx, nc, out, ldo, th, th_out, bad); count_launch();
}

// ---------------------------------------------------------------------------
// Transform builder (thick restart, locking).  Candidates (j x nc, basis
// coordinates, priority order) are orthonormalised by classical Gram-Schmidt
// twice in the j-dimensional coefficient space against the exclusion columns
// (j x ne) and the accepted candidates; a candidate whose remaining norm is
// below 1e-8 is dropped; at most nmax are kept.  Outputs Y (j x jn, basis
// coordinates, ld ldy), *jn_out, and the new frame matrix
// A' = Yh^T A Yh with Yh = S^T Y (jn x jn, ld lda2), i.e. Y^T H Y.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SM_THREADS) k_transform(int j, const double* __restrict__ S, int lds,
                                                          const double* __restrict__ A, int lda,
                                                          const double* __restrict__ cand, int ldc, int nc,
                                                          int nc_a, int lim_a, int a_orth,
                                                          const double* __restrict__ excl, int lde, int ne, int nmax,
                                                          double* __restrict__ Y, int ldy, int* jn_out,
                                                          double* __restrict__ A2, int lda2) {
  extern __shared__ __align__(16) double dsm[];
  double* Ys = dsm;                          // accepted columns (coefficient space)
  double* Yh = Ys + SM_MAXJ * SM_MAXJ;       // S^T Y
  double* AY = Yh + SM_MAXJ * SM_MAXJ;       // A Yh
  __shared__ double v[SM_MAXJ];
  __shared__ double h[2 * SM_MAXJ];
  __shared__ int nacc_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // group A holds Ritz / singular coefficient vectors: when a_orth is set they
  // are orthonormal up to rounding and are copied (up to lim_a of them);
  // otherwise they go through the same Gram-Schmidt as group B
  int c0 = 0;
  if (a_orth) {
    const int na = nc_a < lim_a ? nc_a : lim_a;
    const int na2 = na < nmax ? na : nmax;
    for (int e = tid; e < j * na2; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      Ys[r + c * SM_MAXJ] = cand[r + (size_t)c * ldc];
    }
    if (tid == 0) nacc_s = na2;
    c0 = nc_a;
  } else if (tid == 0) {
    nacc_s = 0;
  }
  __syncthreads();
  // classical Gram-Schmidt twice against [excl | accepted], one warp per inner
  // product, then normalise; a candidate below 1e-8 of its input norm is dropped
  for (int c = c0; c < nc; ++c) {
    const int nacc = nacc_s;
    if (nacc >= nmax) break;
    if (c < nc_a && nacc >= lim_a) continue;  // group A is full: go on with group B
    for (int r = tid; r < j; r += SM_THREADS) v[r] = cand[r + (size_t)c * ldc];
    __syncthreads();
    double n0 = 0.0;
    for (int r = lane; r < j; r += 32) n0 = fma(v[r], v[r], n0);
    n0 = warp_sum(n0);
    const int nb = ne + nacc;
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = warp; q < nb; q += SM_THREADS / 32) {
        const double* col = q < ne ? excl + (size_t)q * lde : Ys + (q - ne) * SM_MAXJ;
        double d = 0.0;
        for (int r = lane; r < j; r += 32) d = fma(col[r], v[r], d);
        d = warp_sum(d);
        if (lane == 0) h[q] = d;
      }
      __syncthreads();
      for (int r = tid; r < j; r += SM_THREADS) {
        double acc = v[r];
        for (int q = 0; q < nb; ++q) {
          const double* col = q < ne ? excl + (size_t)q * lde : Ys + (q - ne) * SM_MAXJ;
          acc = fma(-h[q], col[r], acc);
        }
        v[r] = acc;
      }
      __syncthreads();
    }
    double nv = 0.0;
    for (int r = lane; r < j; r += 32) nv = fma(v[r], v[r], nv);
    nv = sqrt(warp_sum(nv));
    n0 = sqrt(n0);
    if (nv > 1e-8 * (n0 > 1.0 ? 1.0 : n0) && nv > 0.0) {
      for (int r = tid; r < j; r += SM_THREADS) Ys[r + nacc * SM_MAXJ] = v[r] / nv;
      __syncthreads();
      if (tid == 0) nacc_s = nacc + 1;
    }
    __syncthreads();
  }
  // one Newton-Schulz step, Ys <- Ys (3I - Ys^T Ys)/2, removes what rounding
  // left of the loss of orthogonality (so V Y stays orthonormal across restarts)
  {
    const int na = nacc_s;
    double* Gm = Yh;   // scratch: Ys^T Ys, then the copy of Ys
    for (int e = tid; e < na * na; e += SM_THREADS) {
      const int a2 = e % na, c = e / na;
      double d = 0.0;
      for (int r = 0; r < j; ++r) d = fma(Ys[r + a2 * SM_MAXJ], Ys[r + c * SM_MAXJ], d);
      AY[a2 + c * SM_MAXJ] = (a2 == c ? 1.5 : 0.0) - 0.5 * d;
    }
    for (int e = tid; e < j * na; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      Gm[r + c * SM_MAXJ] = Ys[r + c * SM_MAXJ];
    }
    __syncthreads();
    for (int e = tid; e < j * na; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      double acc = 0.0;
      for (int q = 0; q < na; ++q) acc = fma(Gm[r + q * SM_MAXJ], AY[q + c * SM_MAXJ], acc);
      Ys[r + c * SM_MAXJ] = acc;
    }
    __syncthreads();
  }
  const int jn = nacc_s;
  if (A2 == nullptr) {
    for (int e = tid; e < j * jn; e += SM_THREADS) {
      const int r = e % j, c = e / j;
      Y[r + (size_t)c * ldy] = Ys[r + c * SM_MAXJ];
    }
    if (tid == 0) *jn_out = jn;
    return;
  }
  // Yh = S^T Y
  for (int e = tid; e < j * jn; e += SM_THREADS) {
    const int i = e % j, c = e / j;
    double acc = 0.0;
    for (int r = 0; r < j; ++r) acc = fma(S[r + (size_t)i * lds], Ys[r + c * SM_MAXJ], acc);
    Yh[i + c * SM_MAXJ] = acc;
  }
  __syncthreads();
  for (int e = tid; e < j * jn; e += SM_THREADS) {
    const int i = e % j, c = e / j;
    double acc = 0.0;
    for (int r = 0; r < j; ++r) acc = fma(A[i + (size_t)r * lda], Yh[r + c * SM_MAXJ], acc);
    AY[i + c * SM_MAXJ] = acc;
  }
  __syncthreads();
  for (int e = tid; e < jn * jn; e += SM_THREADS) {
    const int a2 = e % jn, c = e / jn;
    if (a2 > c) continue;
    double acc = 0.0;
    for (int r = 0; r < j; ++r) acc = fma(Yh[r + a2 * SM_MAXJ], AY[r + c * SM_MAXJ], acc);
    double acc2 = 0.0;
    for (int r = 0; r < j; ++r) acc2 = fma(Yh[r + c * SM_MAXJ], AY[r + a2 * SM_MAXJ], acc2);
    const double v2 = 0.5 * (acc + acc2);
    A2[a2 + (size_t)c * lda2] = v2;
    A2[c + (size_t)a2 * lda2] = v2;
  }
  for (int e = tid; e < j * jn; e += SM_THREADS) {
    const int r = e % j, c = e / j;
    Y[r + (size_t)c * ldy] = Ys[r + c * SM_MAXJ];
  }
  if (tid == 0) *jn_out = jn;
}

void build_transform(cudaStream_t s, int j, const double* S, int lds, const double* A, int lda, const double* cand,
                     int ldc, int nc, int nc_a, int lim_a, int a_orth, const double* excl, int lde, int ne, int nmax,
                     double* Y, int ldy, int* jn_out, double* A2, int lda2) {
  const size_t smem = sizeof(double) * 3 * SM_MAXJ * SM_MAXJ;
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_transform<<<1, SM_THREADS, smem, s>>>(j, S, lds, A, lda, cand, ldc, nc, nc_a, lim_a, a_orth, excl, lde, ne,
                                          nmax, Y, ldy, jn_out, A2, lda2); count_launch();
}

// QR column bookkeeping of the refined projection: R[0:c, c] = g1 + g2 (the
// two classical Gram-Schmidt passes), R[c, c] = rho = sqrt(tnorm2), zero below;
// the working SVD matrix G gets the same new column and the new row
// [0 ... 0 rho] (G = R S_R with S_R <- blockdiag(S_R, 1)); minv = 1 / rho.
__global__ void k_qr_column(int c, const double* __restrict__ g1, const double* __restrict__ g2,
                            const double* __restrict__ tnorm2, double* R, int ldr, double* G, int ldg, double* SR,
                            int ldsr, double* minv, int update_g) {
  const double rho = sqrt(fmax(tnorm2[0], 0.0));
  for (int r = threadIdx.x; r <= c; r += blockDim.x) {
    const double v = r < c ? (g1 ? g1[r] : 0.0) + (g2 ? g2[r] : 0.0) : rho;
    R[r + (size_t)c * ldr] = v;
    if (update_g) {
      G[r + (size_t)c * ldg] = v;
      if (r < c) {
        G[c + (size_t)r * ldg] = 0.0;
        SR[c + (size_t)r * ldsr] = 0.0;
        SR[r + (size_t)c * ldsr] = 0.0;
      } else {
        SR[c + (size_t)c * ldsr] = 1.0;
      }
    }
  }
  if (threadIdx.x == 0) minv[0] = rho > 0.0 ? 1.0 / rho : 0.0;
}
void qr_column(cudaStream_t s, int c, const double* g1, const double* g2, const double* tnorm2, double* R, int ldr,
               double* G, int ldg, double* SR, int ldsr, double* minv, int update_g) {
  k_qr_column<<<1, SM_MAXJ, 0, s>>>(c, g1, g2, tnorm2, R, ldr, G, ldg, SR, ldsr, minv, update_g); count_launch();
}

// Final triplet of stage 2 from x = [v; u]: out[c] = (||v||^2, ||u||^2) is
// computed elsewhere; here sigma = u^T (A v) / (||u|| ||v||) given the dot.


// Set S (j x j, ld lds) to the identity.
__global__ void k_identity(int j, double* S, int lds) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < j * j; e += blockDim.x * gridDim.x) {
    const int r = e % j, c = e / j;
    S[r + (size_t)c * lds] = r == c ? 1.0 : 0.0;
  }
}
void set_identity(cudaStream_t s, int j, double* S, int lds) { k_identity<<<1, SM_THREADS, 0, s>>>(j, S, lds); count_launch(); }

// ---------------------------------------------------------------------------
// Refined vector of stage 2 by inverse iteration on the triangular factor R
// of W - shift V (Sec. 3.2 needs only the smallest right singular vector of
// R, not the whole SVD): x <- (R^T R)^{-1} x, i.e. a forward solve with R^T
// and a back solve with R, each followed by normalisation, from the start x0
// (the previous refined coordinates; a fixed all-positive vector when x0 is
// null, zero or not finite).  A pivot |r_kk| below 2^-52 max |r_ab| is raised
// to that value, the usual guard of inverse iteration: it only acts when R is
// singular to working precision, and the guarded solve then returns the null
// direction.  The steps stop once rho = ||R x|| falls by less than a relative
// tau, or after maxit steps; the x with the smallest rho is kept.  Each step
// multiplies the components off the smallest singular direction by
// (sigma_min / sigma_2)^2, so near convergence of the outer iteration one
// step settles it.
// One warp; lane l holds rows l and l + 32 (j <= 64).  All branch decisions
// are taken on warp-uniform values (butterfly sums, broadcasts from lane 0).
// Outputs: s1_out (j, unit norm), out[0] = theta1 = s1^T H s1, out[1] = rho,
// steps_out (optional) = steps taken.
// ---------------------------------------------------------------------------
constexpr int RI_LA = SM_MAXJ + 1;

__device__ inline double warp_bcast0(double v) { return __shfl_sync(0xffffffffu, v, 0); }

__global__ void __launch_bounds__(32) k_refined_inv(int j, const double* __restrict__ R, int ldr,
                                                   const double* __restrict__ x0, const double* __restrict__ H,
                                                   int ldh, int maxit, double tau, double* __restrict__ s1_out,
                                                   double* __restrict__ out, int* __restrict__ steps_out) {
  __shared__ double Rs[SM_MAXJ * RI_LA];
  __shared__ double invd[SM_MAXJ];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const int i0 = lane, i1 = lane + 32;
  const bool h0 = i0 < j, h1 = i1 < j;
  double rmax = 0.0;
  for (int e = lane; e < j * j; e += 32) {
    const int r = e % j, c = e / j;
    const double v = r <= c ? R[r + (size_t)c * ldr] : 0.0;
    Rs[r + c * RI_LA] = v;
    rmax = fmax(rmax, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(FULL, rmax, o));
  rmax = warp_bcast0(rmax);
  __syncwarp();
  const double tiny = rmax > 0.0 ? rmax * 0x1p-52 : 1.0;
  for (int i = lane; i < j; i += 32) {
    double d = Rs[i + i * RI_LA];
    if (!(fabs(d) >= tiny)) d = d < 0.0 ? -tiny : tiny;
    invd[i] = 1.0 / d;
  }
  __syncwarp();
  // start vector
  double x_0 = 0.0, x_1 = 0.0;
  if (x0) {
    x_0 = h0 ? x0[i0] : 0.0;
    x_1 = h1 ? x0[i1] : 0.0;
  }
  double nx = warp_bcast0(sqrt(warp_sum(x_0 * x_0 + x_1 * x_1)));
  if (!(nx > 0.0) || !isfinite(nx)) {
    const double g = 0.6180339887498949;
    x_0 = h0 ? 1.0 + (i0 * g - floor(i0 * g)) : 0.0;
    x_1 = h1 ? 1.0 + (i1 * g - floor(i1 * g)) : 0.0;
    nx = warp_bcast0(sqrt(warp_sum(x_0 * x_0 + x_1 * x_1)));
  }
  x_0 /= nx;
  x_1 /= nx;
  // rho(x) = ||R x||
  auto rnorm = [&](double a0, double a1) {
    double w0 = 0.0, w1 = 0.0;
    for (int c = 0; c < j; ++c) {
      const double xc = __shfl_sync(FULL, c < 32 ? a0 : a1, c & 31);
      if (i0 <= c) w0 = fma(Rs[i0 + c * RI_LA], xc, w0);
      if (i1 <= c) w1 = fma(Rs[i1 + c * RI_LA], xc, w1);
    }
    return warp_bcast0(sqrt(warp_sum(w0 * w0 + w1 * w1)));
  };
  double rho = rnorm(x_0, x_1);
  int step = 0;
  while (step < maxit) {
    ++step;
    double b0 = x_0, b1 = x_1;
    // R^T y = x (forward substitution; row k of R is column k of R^T)
    for (int k = 0; k < j; ++k) {
      const double yk = __shfl_sync(FULL, k < 32 ? b0 : b1, k & 31) * invd[k];
      if (lane == (k & 31)) {
        if (k < 32) b0 = yk;
        else b1 = yk;
      }
      if (h0 && i0 > k) b0 = fma(-Rs[k + i0 * RI_LA], yk, b0);
      if (h1 && i1 > k) b1 = fma(-Rs[k + i1 * RI_LA], yk, b1);
    }
    double nb = warp_bcast0(sqrt(warp_sum(b0 * b0 + b1 * b1)));
    if (!(nb > 0.0) || !isfinite(nb)) break;
    b0 /= nb;
    b1 /= nb;
    // R z = y (back substitution)
    for (int k = j - 1; k >= 0; --k) {
      const double zk = __shfl_sync(FULL, k < 32 ? b0 : b1, k & 31) * invd[k];
      if (lane == (k & 31)) {
        if (k < 32) b0 = zk;
        else b1 = zk;
      }
      if (i0 < k) b0 = fma(-Rs[i0 + k * RI_LA], zk, b0);
      if (i1 < k) b1 = fma(-Rs[i1 + k * RI_LA], zk, b1);
    }
    nb = warp_bcast0(sqrt(warp_sum(b0 * b0 + b1 * b1)));
    if (!(nb > 0.0) || !isfinite(nb)) break;
    b0 /= nb;
    b1 /= nb;
    const double rn = rnorm(b0, b1);
    if (!isfinite(rn)) break;
    const bool better = rn < rho;
    const bool stalled = !(rn < rho * (1.0 - tau));
    if (better) {
      x_0 = b0;
      x_1 = b1;
      rho = rn;
    }
    if (stalled) break;
  }
  // theta1 = s1^T H s1
  double a0 = 0.0, a1 = 0.0;
  for (int c = 0; c < j; ++c) {
    const double xc = __shfl_sync(FULL, c < 32 ? x_0 : x_1, c & 31);
    if (h0) a0 = fma(H[i0 + (size_t)c * ldh], xc, a0);
    if (h1) a1 = fma(H[i1 + (size_t)c * ldh], xc, a1);
  }
  const double th = warp_bcast0(warp_sum(x_0 * a0 + x_1 * a1));
  if (h0) s1_out[i0] = x_0;
  if (h1) s1_out[i1] = x_1;
  if (lane == 0) {
    out[0] = th;
    out[1] = rho;
    if (steps_out) *steps_out = step;
  }
}
void refined_inverse(cudaStream_t s, int j, const double* R, int ldr, const double* x0, const double* H, int ldh,
                     int maxit, double tau, double* s1_out, double* out, int* steps_out) {
  ProfScope ps(s, PROF_SMALL);
  k_refined_inv<<<1, 32, 0, s>>>(j, R, ldr, x0, H, ldh, maxit, tau, s1_out, out, steps_out); count_launch();
}

}  // namespace ph
