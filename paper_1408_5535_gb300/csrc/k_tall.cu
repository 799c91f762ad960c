// Tall-skinny dense kernels of the eigensolver iteration: block classical
// Gram-Schmidt passes with the V^T W projection products, basis transforms
// V <- V Y (thick restart / locking), Ritz vectors and residuals
// R = W S - X Theta, and the Jacobi (Olsen) correction.
//
// Storage is T (double, or float in the mixed-precision stage 1); every
// product accumulates per thread in T and across thread blocks in FP64.
// On GB300 the FP64 variants are bound by the FP64 pipe (~1.2 TFLOP/s), the
// FP32 variants by HBM bandwidth.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ph {

static std::atomic<int> g_num_sms{0};
static int num_sms() {
  int v = g_num_sms.load(std::memory_order_relaxed);
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 152;
    g_num_sms.store(v, std::memory_order_relaxed);
  }
  return v;
}

constexpr int CG_ROWS = 256;   // rows per chunk (one per thread in phase A)
constexpr int CG_THREADS = 256;
constexpr int CG_MAXP = 64;    // max basis columns handled per pass
constexpr int CG_PC = CG_MAXP / (CG_THREADS / 32);  // columns per warp

__device__ inline double atomic_add_f64(double* p, double v) { return atomicAdd(p, v); }

__global__ void k_reduce_partials(const double* __restrict__ ws, int blocks, int n1, double* __restrict__ out1,
                                  int n2, double* __restrict__ out2) {
  const int no = n1 + n2;
  const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (o >= no) return;
  double acc = 0.0;
  for (int b = lane; b < blocks; b += 32) acc += ws[(size_t)b * no + o];
  acc = warp_sum(acc);
  if (lane == 0) {
    if (o < n1)
      out1[o] += acc;
    else
      out2[o - n1] += acc;
  }
}
void reduce_partials(cudaStream_t s, RedWs rw, int blocks, int n1, double* out1, int n2, double* out2) {
  const int no = n1 + n2;
  if (!rw.ws || no <= 0) return;
  k_reduce_partials<<<ceil_div(no, 8), 256, 0, s>>>(rw.ws, blocks, n1, out1, n2, out2); count_launch();
}

// 16-byte asynchronous copy global -> shared (no register staging, so a
// thread can keep many in flight), and the wait for all of this thread's.
__device__ inline void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage columns [0, p) of the basis, rows [row0, row0 + rows), into Ps
// (column c at Ps + c * rows): 16-byte asynchronous copies when vec (every
// column start 16-byte aligned) and the chunk lies inside the vectors, else
// element loads with zero fill past n.  Caller synchronises afterwards.
template <typename T>
__device__ inline void stage_cols(const Basis<T>& P, int p, int n, int row0, int rows, bool vec, T* Ps, int tid,
                                  int NT) {
  if (vec && row0 + rows <= n) {
    constexpr int W = 16 / sizeof(T);
    const int segs = rows / W;
    for (int e = tid; e < p * segs; e += NT) {
      const int c = e / segs, sg = e - c * segs;
      const T* src = (c < P.c1 ? P.p1 + (size_t)c * P.ld1 : P.p2 + (size_t)(c - P.c1) * P.ld2) + row0 + sg * W;
      cp_async16(Ps + (size_t)c * rows + sg * W, src);
    }
    cp_async_wait_all();
  } else {
#pragma unroll 4
    for (int e = tid; e < p * rows; e += NT) {
      const int c = e / rows, rr = e - c * rows;
      const int ii = row0 + rr;
      T pc = T(0);
      if (ii < n) pc = c < P.c1 ? P.p1[(size_t)c * P.ld1 + ii] : P.p2[(size_t)(c - P.c1) * P.ld2 + ii];
      Ps[(size_t)c * rows + rr] = pc;
    }
  }
}
template <typename T>
static bool cols16(const T* p, int ld) { return p == nullptr || (((uintptr_t)p & 15) == 0 && (ld * sizeof(T)) % 16 == 0); }

// K consecutive values from 16-byte aligned shared memory, with 16-byte loads.
template <typename T, int K>
__device__ inline void lds_vec(const T* __restrict__ src, T (&d)[K]) {
  if constexpr ((K * sizeof(T)) % 16 == 0) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int u = 0; u < K; u += 4) {
        const float4 t = *reinterpret_cast<const float4*>(src + u);
        d[u] = t.x; d[u + 1] = t.y; d[u + 2] = t.z; d[u + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int u = 0; u < K; u += 2) {
        const double2 t = *reinterpret_cast<const double2*>(src + u);
        d[u] = t.x; d[u + 1] = t.y;
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < K; ++u) d[u] = src[u];
  }
}

// Butterfly reduce-scatter of the N values each lane holds (N a power of two):
// at the level with lane offset O, a lane keeps the half of its live values
// selected by its lane bit O and adds the partner's copy of that half, so a
// warp sum of N values costs N - 1 adds per lane instead of 5 N.  Afterwards
// (N >= 32) lane l holds the warp sums of values l * (N / 32) + u in v[u],
// u < N / 32; (N < 32) v[0] of lane l holds the warp sum of value l / (32 / N).
template <typename T, int N, int O, int CUR>
__device__ __forceinline__ void reduce_scatter_step(T (&v)[N], int lane) {
  if constexpr (O > 0) {
    if constexpr (CUR > 1) {
      constexpr int H = CUR / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const T send = up ? v[i] : v[i + H];
        const T keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      reduce_scatter_step<T, N, O / 2, H>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      reduce_scatter_step<T, N, O / 2, 1>(v, lane);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void reduce_scatter(T (&v)[N], int lane) {
  reduce_scatter_step<T, N, 16, N>(v, lane);
}

// Block CGS pass.  Phase A: all threads load the chunk of P into shared memory
// (independent loads, so short vectors do not wait on one load per column),
// then one thread per row applies T -= P Gsub and stores T.  Phase B: warp w
// accumulates the P^T T entries of columns w, w+8, ... and the T^T T pairs
// k = w, w+8, ...
template <typename T, int Q>
__global__ void __launch_bounds__(CG_THREADS) k_cgs_pass(int n, Basis<T> P, T* __restrict__ Tb, int ldt, int q,
                                                         const double* __restrict__ Gsub, double* __restrict__ Gout,
                                                         double* __restrict__ Tout, int rows, bool vec, RedWs rw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double part[CG_MAXP * 8 + 64];               // the block's Gout and Tout partials
  const int p = P.cols();
  T* Ps = reinterpret_cast<T*>(smem_raw);                 // [p][rows]
  T* Ts = Ps + (size_t)p * rows;                           // [Q][rows]
  T* Gs = Ts + (size_t)Q * rows;                           // [p][Q] row-major, in T precision
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Gs[c * Q + r] = Gsub[c + r * p] (Gsub column-major p x q), zero for r >= q:
  // the Q coefficients of basis column c are contiguous (vector loads)
  if (Gsub)
    for (int k = tid; k < p * Q; k += CG_THREADS) {
      const int c = k / Q, r = k - c * Q;
      Gs[k] = r < q ? (T)Gsub[c + (size_t)r * p] : T(0);
    }
  T accG[CG_PC][Q];
  T accT[(Q * (Q + 1) / 2 + 7) / 8];
#pragma unroll
  for (int a = 0; a < CG_PC; ++a)
#pragma unroll
    for (int r = 0; r < Q; ++r) accG[a][r] = T(0);
#pragma unroll
  for (int a = 0; a < (Q * (Q + 1) / 2 + 7) / 8; ++a) accT[a] = T(0);
  __syncthreads();
  const int nchunks = (n + rows - 1) / rows;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int row0 = ch * rows;
    const int i = row0 + tid;
    const bool act = tid < rows && i < n;
    // ---- phase A
    stage_cols<T>(P, p, n, row0, rows, vec, Ps, tid, CG_THREADS);
    T t[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) t[r] = (act && r < q) ? Tb[(size_t)r * ldt + i] : T(0);
    __syncthreads();
    if (Gsub && tid < rows) {
      for (int c = 0; c < p; ++c) {
        const T pc = Ps[(size_t)c * rows + tid];
#pragma unroll
        {
          T g[Q];
          lds_vec<T, Q>(Gs + (size_t)c * Q, g);
#pragma unroll
          for (int r = 0; r < Q; ++r) t[r] = fma(-pc, g[r], t[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      if (tid < rows) Ts[r * rows + tid] = t[r];
      if (Gsub && act && r < q) Tb[(size_t)r * ldt + i] = t[r];
    }
    __syncthreads();
    // ---- phase B
    if (Gout) {
      // each row of the block is read once from shared memory and used for
      // all of the warp's basis columns (Q + CG_PC loads per Q * CG_PC FMAs)
      for (int rr = lane; rr < rows; rr += 32) {
        T tt[Q];
#pragma unroll
        for (int r = 0; r < Q; ++r) tt[r] = Ts[r * rows + rr];
#pragma unroll
        for (int a = 0; a < CG_PC; ++a) {
          const int c = warp + a * (CG_THREADS / 32);
          if (c < p) {
            const T pv = Ps[(size_t)c * rows + rr];
#pragma unroll
            for (int r = 0; r < Q; ++r) accG[a][r] = fma(pv, tt[r], accG[a][r]);
          }
        }
      }
    }
    if (Tout) {
      int k = 0;
#pragma unroll
      for (int r = 0; r < Q; ++r)
#pragma unroll
        for (int s2 = r; s2 < Q; ++s2, ++k) {
          if (k % 8 == warp) {
            T acc = T(0);
            for (int rr = lane; rr < rows; rr += 32) acc = fma(Ts[r * rows + rr], Ts[s2 * rows + rr], acc);
            accT[k / 8] += acc;
          }
        }
    }
    __syncthreads();
  }
  // ---- reduce within the block (fixed order), then across blocks
  const int n1 = Gout ? p * q : 0, n2 = Tout ? q * q : 0;
  if (Gout) {
    constexpr int NV = CG_PC * Q;
    constexpr int PER = NV >= 32 ? NV / 32 : 1;   // sums held per lane
    constexpr int REP = NV >= 32 ? 1 : 32 / NV;   // lanes holding the same sum
    T (&v)[NV] = reinterpret_cast<T (&)[NV]>(accG);
    reduce_scatter<T, NV>(v, lane);
    if (lane % REP == 0) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int idx = NV >= 32 ? lane * PER + u : lane / REP;
        const int a = idx / Q, r = idx % Q;
        const int c = warp + a * (CG_THREADS / 32);
        if (c < p && r < q) part[c + r * p] = (double)v[u];
      }
    }
  }
  if (Tout) {
    int k = 0;
#pragma unroll
    for (int r = 0; r < Q; ++r)
#pragma unroll
      for (int s2 = r; s2 < Q; ++s2, ++k) {
        if (k % 8 == warp) {
          double v = (double)warp_sum(accT[k / 8]);
          if (lane == 0 && s2 < q) {
            part[n1 + r + s2 * q] = v;
            if (s2 != r) part[n1 + s2 + r * q] = v;
          }
        }
      }
  }
  __syncthreads();
  if (n1 + n2) ordered_commit(part, n1, Gout, n2, Tout, rw);
}

template <typename T, int Q>
static void cgs_launch(cudaStream_t s, int n, const Basis<T>& P, T* Tb, int ldt, int q, const double* Gsub,
                       double* Gout, double* Tout) {
  const int p = P.cols();
  // rows per chunk: 256 when the grid fills the GPU, fewer for short vectors
  // (the FP64 work of a pass then spreads over more SMs)
  int rows = CG_ROWS;
  while (rows > 32 && (int64_t)ceil_div(n, rows) < 2LL * num_sms()) rows >>= 1;
  const size_t smem = sizeof(T) * ((size_t)p * rows + (size_t)Q * rows + (size_t)p * Q);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_cgs_pass<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * ((size_t)CG_MAXP * CG_ROWS + 8 * CG_ROWS + CG_MAXP * 8)));
  });
  int grid = ceil_div(n, rows);
  const int cap = num_sms() * (sizeof(T) == 8 ? 2 : 4);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  const bool vec = cols16(P.p1, P.ld1) && cols16(P.p2, P.ld2);
  const int n1 = (Gout && p > 0) ? p * q : 0, n2 = Tout ? q * q : 0;
  const RedWs rw = red_ws((size_t)grid * (n1 + n2));
  k_cgs_pass<T, Q><<<grid, CG_THREADS, smem, s>>>(n, P, Tb, ldt, q, Gsub, Gout, Tout, rows, vec, rw); count_launch();
  reduce_partials(s, rw, grid, n1, Gout, n2, Tout);
  count_work(pcat<T>(PROF_GRAM),
             2.0 * n * p * q * ((Gsub ? 1 : 0) + (Gout ? 1 : 0)) + (Tout ? (double)n * q * (q + 1) : 0.0),
             (double)sizeof(T) * n * ((Gsub || Gout ? p : 0) + q * (Gsub ? 2 : 1)));
}

template <typename T>
void cgs_pass(cudaStream_t s, int n, const Basis<T>& P, T* Tb, int ldt, int q, const double* Gsub, double* Gout,
              double* Tout) {
  if (n <= 0 || q <= 0) return;
  ProfScope ps(s, pcat<T>(PROF_GRAM));
  Basis<T> PP = P;
  if (PP.cols() == 0) { Gsub = nullptr; Gout = nullptr; }
  switch (q) {
    case 1: cgs_launch<T, 1>(s, n, PP, Tb, ldt, q, Gsub, Gout, Tout); break;
    case 2: cgs_launch<T, 2>(s, n, PP, Tb, ldt, q, Gsub, Gout, Tout); break;
    case 3: case 4: cgs_launch<T, 4>(s, n, PP, Tb, ldt, q, Gsub, Gout, Tout); break;
    default: cgs_launch<T, 8>(s, n, PP, Tb, ldt, q, Gsub, Gout, Tout); break;
  }
}

// ---------------------------------------------------------------------------
// Out = P * Y [- Xs diag(theta)], optional column norms.
// ---------------------------------------------------------------------------
constexpr int TS_ROWS = 128;
constexpr int TS_CB = 8;       // output columns per pass of k_tall_small
template <typename T>
__global__ void __launch_bounds__(TS_ROWS) k_tall_small(int n, const T* P, int ldp, int p,
                                                        const double* __restrict__ Y, int ldy, int r, T* Out,
                                                        int ldo, const T* __restrict__ Xs, int ldx,
                                                        const double* __restrict__ theta, double* norms2, bool vec,
                                                        RedWs rw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double wn[64][TS_ROWS / 32];                 // per-warp partial norms (fixed order)
  const int rp = (r + TS_CB - 1) / TS_CB * TS_CB;                 // r padded to whole column blocks
  double* nrm = reinterpret_cast<double*>(smem_raw);            // [r]
  T* Ys = reinterpret_cast<T*>(smem_raw + sizeof(double) * (size_t)((r + 1) & ~1));  // [p][rp] row-major
  T* Ps = Ys + (size_t)p * rp;                                   // [p][blockDim.x], 16-byte aligned
  const int tid = threadIdx.x;
  for (int k = tid; k < p * rp; k += blockDim.x) {
    const int a = k / rp, c = k - a * rp;
    Ys[k] = c < r ? (T)Y[a + (size_t)c * ldy] : T(0);
  }
  if (norms2)
    for (int c = tid; c < 64 * (TS_ROWS / 32); c += blockDim.x) wn[c / (TS_ROWS / 32)][c % (TS_ROWS / 32)] = 0.0;
  __syncthreads();
  const int R = blockDim.x;
  const int nchunks = (n + R - 1) / R;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int i = ch * R + tid;
    const bool act = i < n;
    Basis<T> PB{P, ldp, p, nullptr, 0, 0};
    stage_cols<T>(PB, p, n, ch * R, R, vec, Ps, tid, R);
    __syncthreads();  // every row of the chunk is read before any (in-place) write
    // TS_CB output columns at a time: one shared load of the row's basis
    // value and vector loads of the block's coefficients per TS_CB FMAs
    for (int c0 = 0; c0 < r; c0 += TS_CB) {
      const int nc = r - c0 < TS_CB ? r - c0 : TS_CB;
      T acc[TS_CB];
#pragma unroll
      for (int u = 0; u < TS_CB; ++u) acc[u] = T(0);
      for (int a = 0; a < p; ++a) {
        const T pa = Ps[(size_t)a * R + tid];
        T yv[TS_CB];
        lds_vec<T, TS_CB>(Ys + (size_t)a * rp + c0, yv);
#pragma unroll
        for (int u = 0; u < TS_CB; ++u) acc[u] = fma(pa, yv[u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < TS_CB; ++u) {
        if (u < nc) {
          const int c = c0 + u;
          T o = acc[u];
          if (theta && act) o = fma((T)(-theta[c]), Xs[(size_t)c * ldx + i], o);
          if (act) Out[(size_t)c * ldo + i] = o;
          if (norms2) {
            double v = warp_sum((double)o * (double)o);
            if ((tid & 31) == 0) wn[c][tid >> 5] += v;
          }
        }
      }
    }
    __syncthreads();
  }
  if (norms2) {
    __syncthreads();
    for (int c = tid; c < r; c += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wn[c][w];
      nrm[c] = t;
    }
    __syncthreads();
    ordered_commit(nrm, r, norms2, 0, nullptr, rw);
  }
}

template <typename T>
void tall_times_small(cudaStream_t s, int n, const T* P, int ldp, int p, const double* Y, int ldy, int r, T* Out,
                      int ldo, const T* Xs, int ldx, const double* theta, double* norms2) {
  if (n <= 0 || r <= 0) return;
  ProfScope ps(s, pcat<T>(PROF_TALL));
  int R = TS_ROWS;
  while (R > 32 && (int64_t)ceil_div(n, R) < 2LL * num_sms()) R >>= 1;
  const int rp = (r + TS_CB - 1) / TS_CB * TS_CB;
  const size_t smem = sizeof(double) * (size_t)((r + 1) & ~1) + sizeof(T) * ((size_t)p * rp + (size_t)p * R);
  static std::atomic<uint64_t> attr_done{0};
  once_per_device(attr_done, [&] {
    cudaFuncSetAttribute(k_tall_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  int grid = ceil_div(n, R);
  const int cap = num_sms() * 8;
  if (grid > cap) grid = cap;
  const RedWs rw = norms2 ? red_ws((size_t)grid * r) : RedWs{};
  k_tall_small<T><<<grid, R, smem, s>>>(n, P, ldp, p, Y, ldy, r, Out, ldo, Xs, ldx, theta, norms2,
                                        cols16(P, ldp), rw); count_launch();
  if (norms2) reduce_partials(s, rw, grid, r, norms2, 0, nullptr);
  count_work(pcat<T>(PROF_TALL), 2.0 * n * p * r + (theta ? 2.0 * n * r : 0.0) + (norms2 ? 2.0 * n * r : 0.0),
             (double)sizeof(T) * n * (p + r + (theta ? r : 0)));
}

// ---------------------------------------------------------------------------
// T <- T * M (q x q, FP64), optional copy to Dst.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scale_block(int n, T* Tb, int ldt, int q, const double* __restrict__ M, T* Dst, int ldd) {
  __shared__ T Ms[64];
  for (int k = threadIdx.x; k < q * q; k += blockDim.x) Ms[k] = (T)M[k];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T t[8], o[8];
  for (int r = 0; r < q; ++r) t[r] = Tb[(size_t)r * ldt + i];
  for (int c = 0; c < q; ++c) {
    T acc = T(0);
    for (int r = 0; r < q; ++r) acc = fma(t[r], Ms[r + c * q], acc);
    o[c] = acc;
  }
  for (int c = 0; c < q; ++c) {
    Tb[(size_t)c * ldt + i] = o[c];
    if (Dst) Dst[(size_t)c * ldd + i] = o[c];
  }
}
template <typename T>
void scale_block(cudaStream_t s, int n, T* Tb, int ldt, int q, const double* M, T* Dst, int ldd) {
  if (n > 0 && q > 0) k_scale_block<T><<<ceil_div(n, 256), 256, 0, s>>>(n, Tb, ldt, q, M, Dst, ldd); count_launch();
}

template <typename T>
__global__ void k_cm_to_rm(int n, const T* __restrict__ src, int lds, int q, T* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int r = 0; r < q; ++r) dst[(size_t)i * q + r] = src[(size_t)r * lds + i];
}
template <typename T>
__global__ void k_rm_to_cm(int n, const T* __restrict__ src, int q, T* __restrict__ dst, int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int r = 0; r < q; ++r) dst[(size_t)r * ldd + i] = src[(size_t)i * q + r];
}
template <typename T> void cm_to_rm(cudaStream_t s, int n, const T* src, int lds, int q, T* dst) {
  if (n > 0 && q > 0) k_cm_to_rm<T><<<ceil_div(n, 256), 256, 0, s>>>(n, src, lds, q, dst); count_launch();
}
template <typename T> void rm_to_cm(cudaStream_t s, int n, const T* src, int q, T* dst, int ldd) {
  if (n > 0 && q > 0) k_rm_to_cm<T><<<ceil_div(n, 256), 256, 0, s>>>(n, src, q, dst, ldd); count_launch();
}

// ---------------------------------------------------------------------------
// Jacobi (diag(C) - theta)^-1 with the Olsen correction.
// ---------------------------------------------------------------------------
__device__ inline double guarded(double d, double guard) {
  if (fabs(d) < guard) return d < 0 ? -guard : guard;
  return d;
}
template <typename T>
__global__ void k_jacobi_dots(int n, const double* __restrict__ d, const T* __restrict__ X, int ldx,
                              const T* __restrict__ R, int ldr, int q, const double* __restrict__ theta, double guard,
                              double* dots, RedWs rw) {
  __shared__ double wp[16][8];
  __shared__ double part[16];
  double a[8], b[8];
  for (int c = 0; c < q; ++c) a[c] = b[c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int c = 0; c < q; ++c) {
      const double m = 1.0 / guarded(d[i] - theta[c], guard);
      const double x = (double)X[(size_t)c * ldx + i];
      a[c] += x * m * (double)R[(size_t)c * ldr + i];
      b[c] += x * m * x;
    }
  }
  for (int c = 0; c < q; ++c) {
    double va = warp_sum(a[c]), vb = warp_sum(b[c]);
    if ((threadIdx.x & 31) == 0) {
      wp[2 * c][threadIdx.x >> 5] = va;
      wp[2 * c + 1][threadIdx.x >> 5] = vb;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * q) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wp[threadIdx.x][w];
    part[threadIdx.x] = t;
  }
  __syncthreads();
  ordered_commit(part, 2 * q, dots, 0, nullptr, rw);
}
template <typename T>
__global__ void k_jacobi_apply(int n, const double* __restrict__ d, const T* __restrict__ X, int ldx,
                               const T* __restrict__ R, int ldr, int q, const double* __restrict__ theta, double guard,
                               const double* __restrict__ dots, T* __restrict__ Tout, int ldt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < q; ++c) {
    const double m = 1.0 / guarded(d[i] - theta[c], guard);
    const double e = dots[2 * c + 1] != 0.0 ? dots[2 * c] / dots[2 * c + 1] : 0.0;
    Tout[(size_t)c * ldt + i] = (T)(m * ((double)R[(size_t)c * ldr + i] - e * (double)X[(size_t)c * ldx + i]));
  }
}
template <typename T>
void jacobi_dots(cudaStream_t s, int n, const double* d, const T* X, int ldx, const T* R, int ldr, int q,
                 const double* theta, double guard, double* dots) {
  int grid = ceil_div(n, 256);
  if (grid > num_sms() * 4) grid = num_sms() * 4;
  if (n <= 0) return;
  const RedWs rw = red_ws((size_t)grid * 2 * q);
  k_jacobi_dots<T><<<grid, 256, 0, s>>>(n, d, X, ldx, R, ldr, q, theta, guard, dots, rw); count_launch();
  reduce_partials(s, rw, grid, 2 * q, dots, 0, nullptr);
}
template <typename T>
void jacobi_apply(cudaStream_t s, int n, const double* d, const T* X, int ldx, const T* R, int ldr, int q,
                  const double* theta, double guard, const double* dots, T* Tout, int ldt) {
  if (n > 0) k_jacobi_apply<T><<<ceil_div(n, 256), 256, 0, s>>>(n, d, X, ldx, R, ldr, q, theta, guard, dots, Tout, ldt); count_launch();
}

template <typename T>
__global__ void k_fill_random(int n, T* dst, uint64_t seed, uint64_t stream) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)sm64_pm1(seed, stream, (uint64_t)i);
}
template <typename T> void fill_random(cudaStream_t s, int n, T* dst, uint64_t seed, uint64_t stream) {
  if (n > 0) k_fill_random<T><<<ceil_div(n, 256), 256, 0, s>>>(n, dst, seed, stream); count_launch();
}

__global__ void k_f32_f64(int64_t n, const float* a, double* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void k_f64_f32(int64_t n, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
void convert_f32_to_f64(cudaStream_t s, int64_t n, const float* a, double* b) {
  if (n > 0) k_f32_f64<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, a, b); count_launch();
}
void convert_f64_to_f32(cudaStream_t s, int64_t n, const double* a, float* b) {
  if (n > 0) k_f64_f32<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, a, b); count_launch();
}
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
void axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y) {
  if (n > 0) k_axpby<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, a, x, b, y); count_launch();
}

template <typename T>
__global__ void k_colnorms(int n, const T* __restrict__ X, int ldx, int q, double* norms2, RedWs rw) {
  __shared__ double wp[8][8];
  __shared__ double part[8];
  double a[8];
  for (int c = 0; c < q; ++c) a[c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < q; ++c) {
      const double v = (double)X[(size_t)c * ldx + i];
      a[c] += v * v;
    }
  for (int c = 0; c < q; ++c) {
    double v = warp_sum(a[c]);
    if ((threadIdx.x & 31) == 0) wp[c][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < q) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wp[threadIdx.x][w];
    part[threadIdx.x] = t;
  }
  __syncthreads();
  ordered_commit(part, q, norms2, 0, nullptr, rw);
}
template <typename T> void col_norms2_dense(cudaStream_t s, int n, const T* X, int ldx, int q, double* norms2) {
  int grid = ceil_div(n, 256);
  if (grid > num_sms() * 4) grid = num_sms() * 4;
  if (n <= 0) return;
  const RedWs rw = red_ws((size_t)grid * q);
  k_colnorms<T><<<grid, 256, 0, s>>>(n, X, ldx, q, norms2, rw); count_launch();
  reduce_partials(s, rw, grid, q, norms2, 0, nullptr);
}

// out[0] += x^T y (FP64)
__global__ void k_dot(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* out, RedWs rw) {
  __shared__ double wp[8];
  __shared__ double part[1];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a = fma(x[i], y[i], a);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wp[w];
    part[0] = t;
  }
  __syncthreads();
  ordered_commit(part, 1, out, 0, nullptr, rw);
}
void dot_accum(cudaStream_t s, int64_t n, const double* x, const double* y, double* out) {
  int grid = ceil_div(n, 256);
  if (grid > num_sms() * 4) grid = num_sms() * 4;
  if (n <= 0) return;
  const RedWs rw = red_ws((size_t)grid);
  k_dot<<<grid, 256, 0, s>>>(n, x, y, out, rw); count_launch();
  reduce_partials(s, rw, grid, 1, out, 0, nullptr);
}
// y = x / d elementwise; a |d| below guard is raised to +-guard (guard 0: none)
__global__ void k_diag_div(int64_t n, const double* __restrict__ x, const double* __restrict__ d, double guard,
                           double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double di = d[i];
    if (fabs(di) < guard) di = di < 0 ? -guard : guard;
    y[i] = x[i] / di;
  }
}
void diag_div(cudaStream_t s, int64_t n, const double* x, const double* d, double guard, double* y) {
  int grid = ceil_div(n, 256);
  if (grid > num_sms() * 8) grid = num_sms() * 8;
  if (n > 0) k_diag_div<<<grid, 256, 0, s>>>(n, x, d, guard, y); count_launch();
}
// out = a - (dots[0] / dots[1]) b, or a when dots[1] == 0 (the Olsen form)
__global__ void k_olsen_combine(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                const double* __restrict__ dots, double* __restrict__ out) {
  const double e = dots[1] != 0.0 ? dots[0] / dots[1] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fma(-e, b[i], a[i]);
}
void olsen_combine(cudaStream_t s, int64_t n, const double* a, const double* b, const double* dots, double* out) {
  int grid = ceil_div(n, 256);
  if (grid > num_sms() * 8) grid = num_sms() * 8;
  if (n > 0) k_olsen_combine<<<grid, 256, 0, s>>>(n, a, b, dots, out); count_launch();
}
__global__ void k_square(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * x[i];
}
void square(cudaStream_t s, int64_t n, const double* x, double* y) {
  if (n > 0) k_square<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, x, y); count_launch();
}

// x *= a (a read from device memory when ap != nullptr)
__global__ void k_scal(int64_t n, double a, const double* ap, double* x) {
  const double f = ap ? ap[0] : a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}
void scal(cudaStream_t s, int64_t n, double a, const double* ap, double* x) {
  if (n > 0) k_scal<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, a, ap, x); count_launch();
}
// x[i] = v (constant fill)
template <typename T>
__global__ void k_fill(int64_t n, T v, T* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}
template <typename T> void fill_const(cudaStream_t s, int64_t n, T v, T* x) {
  if (n > 0) k_fill<T><<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, v, x); count_launch();
}
template void fill_const<double>(cudaStream_t, int64_t, double, double*);
template void fill_const<float>(cudaStream_t, int64_t, float, float*);

// explicit instantiations
#define PH_INST(T)                                                                                              \
  template void cgs_pass<T>(cudaStream_t, int, const Basis<T>&, T*, int, int, const double*, double*, double*); \
  template void tall_times_small<T>(cudaStream_t, int, const T*, int, int, const double*, int, int, T*, int,    \
                                    const T*, int, const double*, double*);                                    \
  template void scale_block<T>(cudaStream_t, int, T*, int, int, const double*, T*, int);                       \
  template void cm_to_rm<T>(cudaStream_t, int, const T*, int, int, T*);                                        \
  template void rm_to_cm<T>(cudaStream_t, int, const T*, int, T*, int);                                        \
  template void jacobi_dots<T>(cudaStream_t, int, const double*, const T*, int, const T*, int, int,            \
                               const double*, double, double*);                                                \
  template void jacobi_apply<T>(cudaStream_t, int, const double*, const T*, int, const T*, int, int,           \
                                const double*, double, const double*, T*, int);                                \
  template void fill_random<T>(cudaStream_t, int, T*, uint64_t, uint64_t);                                     \
  template void col_norms2_dense<T>(cudaStream_t, int, const T*, int, int, double*);
PH_INST(double)
PH_INST(float)

}  // namespace ph

namespace ph {

// ---------------------------------------------------------------------------
// Conjugate gradients on (A^T A - shift I) x = r for up to 8 right-hand sides
// in lockstep: row-major n x b blocks, per-column FP64 scalars on the device
// (rr = ||r||^2, rrn = the next ||r||^2, pq = p^T q, act = still iterating).
// ---------------------------------------------------------------------------
template <int B>
__device__ inline void block_reduce_add(double (&v)[B], double* out, int b) {
  __shared__ double red[8][B];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < B; ++c) v[c] = warp_sum(v[c]);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < B; ++c) red[w][c] = v[c];
  __syncthreads();
  if (threadIdx.x < b) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
    atomicAdd(out + threadIdx.x, s);
  }
}

// q <- q - shift p; pq[c] += p_c^T q_c
__global__ void __launch_bounds__(256) k_cg_pq(int n, int b, double shift, const double* __restrict__ P,
                                               double* __restrict__ Q, double* __restrict__ pq) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < b; ++c) {
      const size_t k = (size_t)i * b + c;
      const double q = Q[k] - shift * P[k];
      Q[k] = q;
      acc[c] += P[k] * q;
    }
  block_reduce_add<8>(acc, pq, b);
}

// alpha = rr / pq; x += alpha p; r -= alpha q; rrn[c] += ||r_c||^2
__global__ void __launch_bounds__(256) k_cg_update(int n, int b, const double* __restrict__ P,
                                                   const double* __restrict__ Q, double* __restrict__ X,
                                                   double* __restrict__ R, const double* __restrict__ rr,
                                                   const double* __restrict__ pq, const int* __restrict__ act,
                                                   double* __restrict__ rrn) {
  double al[8], acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < b; ++c) al[c] = (act[c] && pq[c] > 0.0) ? rr[c] / pq[c] : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < b; ++c) {
      const size_t k = (size_t)i * b + c;
      X[k] += al[c] * P[k];
      const double r = R[k] - al[c] * Q[k];
      R[k] = r;
      acc[c] += r * r;
    }
  block_reduce_add<8>(acc, rrn, b);
}

// beta = rrn / rr; p = r + beta p (active columns)
__global__ void __launch_bounds__(256) k_cg_dir(int n, int b, const double* __restrict__ R, double* __restrict__ P,
                                                const double* __restrict__ rr, const double* __restrict__ rrn,
                                                const int* __restrict__ act) {
  double be[8];
  for (int c = 0; c < b; ++c) be[c] = (act[c] && rr[c] > 0.0) ? rrn[c] / rr[c] : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int c = 0; c < b; ++c) {
      if (!act[c]) continue;
      const size_t k = (size_t)i * b + c;
      P[k] = R[k] + be[c] * P[k];
    }
}

// per column: count the iteration, rr <- rrn, stop when rr <= tol2 rr0 (or a
// non-positive curvature p^T q <= 0), clear the accumulators
__global__ void k_cg_next(int b, double* rr, double* rrn, const double* rr0, double tol2, double* pq, int* act,
                          int* iters, int* bad) {
  const int c = threadIdx.x;
  if (c >= b) return;
  if (act[c]) {
    iters[c] += 1;
    if (!(pq[c] > 0.0)) bad[0] = 1;
    rr[c] = rrn[c];
    act[c] = (pq[c] > 0.0 && rrn[c] > tol2 * rr0[c]) ? 1 : 0;
  }
  rrn[c] = 0.0;
  pq[c] = 0.0;
}

void cg_pq(cudaStream_t s, int n, int b, double shift, const double* P, double* Q, double* pq) {
  k_cg_pq<<<std::min(ceil_div(n, 256), 4 * num_sms()), 256, 0, s>>>(n, b, shift, P, Q, pq);
  count_launch();
}
void cg_update(cudaStream_t s, int n, int b, const double* P, const double* Q, double* X, double* R,
               const double* rr, const double* pq, const int* act, double* rrn) {
  k_cg_update<<<std::min(ceil_div(n, 256), 4 * num_sms()), 256, 0, s>>>(n, b, P, Q, X, R, rr, pq, act, rrn);
  count_launch();
}
void cg_dir(cudaStream_t s, int n, int b, const double* R, double* P, const double* rr, const double* rrn,
            const int* act) {
  k_cg_dir<<<std::min(ceil_div(n, 256), 4 * num_sms()), 256, 0, s>>>(n, b, R, P, rr, rrn, act);
  count_launch();
}
void cg_next(cudaStream_t s, int b, double* rr, double* rrn, const double* rr0, double tol2, double* pq, int* act,
             int* iters, int* bad) {
  k_cg_next<<<1, 32, 0, s>>>(b, rr, rrn, rr0, tol2, pq, act, iters, bad);
  count_launch();
}

}  // namespace ph
