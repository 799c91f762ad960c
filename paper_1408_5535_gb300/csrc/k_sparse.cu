// Sparse kernels: products with C = A^T A and B = [0 A^T; A 0] (Section 1 of the
// PHSVDS paper), the CSR -> CSC transpose they use, and diag(C).
//
// Layout: CSR of A (row_ptr int32, col int32, val T); the CSC copy is the CSR of
// A^T.  Blocks of b vectors are ROW-major n x b (the b values of a row are
// contiguous, so one gathered row is one 8..64-byte vector load).
#include "common.cuh"
#include "kernels.h"

namespace ph {

// 256-bit gather of one 32-byte row (8 floats or 4 doubles); p must be
// 32-byte aligned.  Read-only path: X is not written by the kernel.  NA: do
// not allocate the row in L1 (rows of an unstructured matrix are rarely
// re-read by the same SM; skipping L1 keeps its lines for the index stream).
template <typename T, int B, bool NA>
__device__ inline void load_row_256(const T* p, T (&r)[B]) {
  static_assert(sizeof(T) * B == 32, "32-byte rows only");
  if constexpr (sizeof(T) == 4) {
    if constexpr (NA)
      asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
                   : "l"(p));
    else
      asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
                   : "l"(p));
  } else {
    if constexpr (NA)
      asm volatile("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                   : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3])
                   : "l"(p));
    else
      asm volatile("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
                   : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3])
                   : "l"(p));
  }
}

// Loads of the matrix stream (indices, values): L1-allocating, so the
// sector shared by consecutive slot loads of a row is fetched from L2 once,
// with an L2 evict-first policy (the matrix is read once per product and
// should not push the gathered rows out of L2).
__device__ inline uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ inline int ld_stream(const int* p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ inline float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ inline double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

// Gathers of the U rows X(col[u], :) whose slot is live; a dead slot issues
// no load (so it costs no L1 wavefront) and contributes zeros.  W: rows are 32
// bytes and X is 32-byte aligned -> one 256-bit load per row.
template <typename T, int B, int U, bool W, bool NA>
__device__ inline void gather_rows(const T* __restrict__ X, const int (&col)[U], const bool (&ok)[U], T (&x)[U][B]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (ok[u]) {
      if constexpr (W)
        load_row_256<T, B, NA>(X + (size_t)col[u] * B, x[u]);
      else
        load_row<T, B>(X + (size_t)col[u] * B, x[u]);
    } else {
#pragma unroll
      for (int q = 0; q < B; ++q) x[u][q] = T(0);
    }
  }
}

// Loads U (column, value) slots of one row for this lane: slot u is entry
// base + u*L + lane.  Every address stays inside the row (e0 < e1 here): a
// dead slot re-reads entry e0 and is marked not live; a column index outside
// [0, xrows) is never gathered (guard against a corrupted index).
template <typename T, int L, int U>
__device__ inline void load_slots(const int* __restrict__ ci, const T* __restrict__ va, int base, int lane, int e0,
                                  int e1, int xrows, uint64_t pol, int (&col)[U], T (&v)[U], bool (&ok)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int e = base + u * L + lane;
    const bool live = e < e1;
    const int ec = live ? e : e0;
    const int c = ld_stream(ci + ec, pol);
    const bool inr = (unsigned)c < (unsigned)xrows;
    ok[u] = live && inr;
    col[u] = inr ? c : 0;
    const T a = ld_stream(va + ec, pol);
    v[u] = ok[u] ? a : T(0);
  }
}

// Z = A X: one group of L lanes per sparse row.  Each pass a lane loads U
// (column, value) slots (streaming loads: the matrix is read once and should
// not evict the gathered rows from L2), then issues the live gathers back to
// back so up to U independent loads are in flight per lane; the B partial
// sums are reduced inside the group at the end.
template <typename T, int B, int L, int U, bool W, bool NA>
__global__ void __launch_bounds__(256) k_csr_rows(int nrows, int xrows, const int* __restrict__ rp,
                                                  const int* __restrict__ ci, const T* __restrict__ va,
                                                  const T* __restrict__ X, T* __restrict__ Z) {
  const int lane = threadIdx.x % L;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / L;
  const bool active = row < nrows;  // inactive groups still take part in the shuffles
  T acc[B];
#pragma unroll
  for (int q = 0; q < B; ++q) acc[q] = T(0);
  const int e0 = active ? rp[row] : 0, e1 = active ? rp[row + 1] : 0;
  const uint64_t pol = l2_evict_first_policy();
  for (int base = e0; base < e1; base += L * U) {
    int col[U];
    T v[U];
    bool ok[U];
    load_slots<T, L, U>(ci, va, base, lane, e0, e1, xrows, pol, col, v, ok);
    T x[U][B];
    gather_rows<T, B, U, W, NA>(X, col, ok, x);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < B; ++q) acc[q] = fma(v[u], x[u][q], acc[q]);
  }
  if constexpr (L > 1) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < B; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, L);
  }
  if (active && lane == 0) store_row<T, B>(Z + (size_t)row * B, acc);
}

// Fused single pass Y += A^T (A X): a group computes z = a_i^T X for its row
// (same slots and gathers as above), keeps it in registers and scatters
// a_ij * z into Y with L2 atomics (128-bit vector atomics for FP32).  A row
// that fits in one pass (length <= L*U) scatters from the slots already in
// registers; longer rows re-read their entries.
template <typename T, int B, int L, int U, bool W, bool NA>
__global__ void __launch_bounds__(256) k_ata_fused(int nrows, int xrows, const int* __restrict__ rp,
                                                   const int* __restrict__ ci, const T* __restrict__ va,
                                                   const T* __restrict__ X, T* __restrict__ Y) {
  const int lane = threadIdx.x % L;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / L;
  const bool active = row < nrows;
  T z[B];
#pragma unroll
  for (int q = 0; q < B; ++q) z[q] = T(0);
  const int e0 = active ? rp[row] : 0, e1 = active ? rp[row + 1] : 0;
  int col[U];
  T v[U];
  bool ok[U];
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = false;
  const uint64_t pol = l2_evict_first_policy();
  for (int base = e0; base < e1; base += L * U) {
    load_slots<T, L, U>(ci, va, base, lane, e0, e1, xrows, pol, col, v, ok);
    T x[U][B];
    gather_rows<T, B, U, W, NA>(X, col, ok, x);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < B; ++q) z[q] = fma(v[u], x[u][q], z[q]);
  }
  if constexpr (L > 1) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < B; ++q) z[q] += __shfl_xor_sync(0xffffffffu, z[q], o, L);
  }
  if (e1 - e0 <= L * U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      T y[B];
#pragma unroll
      for (int q = 0; q < B; ++q) y[q] = v[u] * z[q];
      atomic_add_row<T, B>(Y + (size_t)col[u] * B, y);
    }
    return;
  }
  for (int e = e0 + lane; e < e1; e += L) {
    const int c = ci[e];
    if ((unsigned)c >= (unsigned)xrows) continue;
    const T a = va[e];
    T y[B];
#pragma unroll
    for (int q = 0; q < B; ++q) y[q] = a * z[q];
    atomic_add_row<T, B>(Y + (size_t)c * B, y);
  }
}

// U (loads in flight per lane): 4, or 2 for 8-wide FP64 rows (register budget)
template <typename T, int B> constexpr int unroll_for() { return (sizeof(T) == 8 && B == 8) ? 2 : 4; }

// wide (256-bit) gathers apply to 32-byte rows of a 32-byte aligned block
template <typename T, int B> constexpr bool wide_rows() { return sizeof(T) * B == 32; }
template <typename T> static bool aligned32(const T* p) { return ((uintptr_t)p & 31) == 0; }

template <typename T, int B, bool FUSED, int L>
static void launch_rows(cudaStream_t s, int nrows, int xrows, const int* rp, const int* ci, const T* va, const T* X,
                        T* out, bool l1_gather) {
  const int th = 256;
  const int blocks = ceil_div((int64_t)nrows * L, th);
  constexpr int U = unroll_for<T, B>();
  if constexpr (wide_rows<T, B>()) {
    if (aligned32(X)) {
      if (l1_gather) {
        if constexpr (FUSED)
          k_ata_fused<T, B, L, U, true, false><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
        else
          k_csr_rows<T, B, L, U, true, false><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
      } else {
        if constexpr (FUSED)
          k_ata_fused<T, B, L, U, true, true><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
        else
          k_csr_rows<T, B, L, U, true, true><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
      }
      count_launch();
      return;
    }
  }
  if constexpr (FUSED)
    k_ata_fused<T, B, L, U, false, false><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
  else
    k_csr_rows<T, B, L, U, false, false><<<blocks, th, 0, s>>>(nrows, xrows, rp, ci, va, X, out);
  count_launch();
}

template <typename T, int B, bool FUSED>
static void dispatch_L(cudaStream_t s, int L, int nrows, int xrows, const int* rp, const int* ci, const T* va,
                       const T* X, T* out, bool l1) {
  if (nrows <= 0) return;
  switch (L) {
    case 1: launch_rows<T, B, FUSED, 1>(s, nrows, xrows, rp, ci, va, X, out, l1); break;
    case 2: launch_rows<T, B, FUSED, 2>(s, nrows, xrows, rp, ci, va, X, out, l1); break;
    case 4: launch_rows<T, B, FUSED, 4>(s, nrows, xrows, rp, ci, va, X, out, l1); break;
    case 8: launch_rows<T, B, FUSED, 8>(s, nrows, xrows, rp, ci, va, X, out, l1); break;
    default: launch_rows<T, B, FUSED, 16>(s, nrows, xrows, rp, ci, va, X, out, l1); break;
  }
}

// lanes: group width; a negative value -l means width l with the row
// gathers not allocated in L1 (32-byte rows only).
template <typename T, bool FUSED>
static void dispatch_B(cudaStream_t s, int b, int lanes, const SparseView<T>& A, const T* X, T* out) {
  const bool l1 = lanes > 0;
  const int L = lanes > 0 ? lanes : -lanes;
  switch (b) {
    case 1: dispatch_L<T, 1, FUSED>(s, L, A.nrows, A.ncols, A.ptr, A.idx, A.val, X, out, l1); break;
    case 2: dispatch_L<T, 2, FUSED>(s, L, A.nrows, A.ncols, A.ptr, A.idx, A.val, X, out, l1); break;
    case 4: dispatch_L<T, 4, FUSED>(s, L, A.nrows, A.ncols, A.ptr, A.idx, A.val, X, out, l1); break;
    case 8: dispatch_L<T, 8, FUSED>(s, L, A.nrows, A.ncols, A.ptr, A.idx, A.val, X, out, l1); break;
    default: break;
  }
}

int lanes_for(double avg_row) {
  if (avg_row <= 2.5) return 1;
  if (avg_row <= 6.0) return 2;
  if (avg_row <= 16.0) return 4;
  return 8;
}

// Algorithmic work of one product with C = A^T A on b vectors (the SpMM unit):
// one read of the CSR (values and column indices, row offsets), X read once,
// Y written once; 4 nnz b flops.
template <typename T>
static void count_ata(const SparseView<T>& A, int ncols, int b) {
  count_work(pcat<T>(PROF_CSPMM), 4.0 * (double)A.nnz * b,
             (double)A.nnz * (sizeof(T) + 4) + 4.0 * (A.nrows + 1) + 2.0 * sizeof(T) * ncols * b);
}

template <typename T>
void csr_spmm(cudaStream_t s, const SparseView<T>& A, int b, const T* X, T* Z, int lanes) {
  ProfScope ps(s, pcat<T>(PROF_SPMV));
  count_work(pcat<T>(PROF_SPMV), 2.0 * (double)A.nnz * b,
             (double)A.nnz * (sizeof(T) + 4) + 4.0 * (A.nrows + 1) + (double)sizeof(T) * b * (A.ncols + A.nrows));
  dispatch_B<T, false>(s, b, lanes != 0 ? lanes : lanes_for(A.avg_row()), A, X, Z);
}

template <typename T>
void ata_fused(cudaStream_t s, const SparseView<T>& A, int ncols, int b, const T* X, T* Y, int lanes) {
  ProfScope ps(s, pcat<T>(PROF_CSPMM));
  count_ata(A, ncols, b);
  cudaMemsetAsync(Y, 0, sizeof(T) * (size_t)ncols * b, s);
  dispatch_B<T, true>(s, b, lanes != 0 ? lanes : lanes_for(A.avg_row()), A, X, Y);
}

template <typename T>
void ata_two_phase(cudaStream_t s, const SparseView<T>& A, const SparseView<T>& At, int b, const T* X, T* Y,
                   T* Z, int lanes_a, int lanes_at) {
  ProfScope ps(s, pcat<T>(PROF_CSPMM));
  count_ata(A, At.nrows, b);
  dispatch_B<T, false>(s, b, lanes_a != 0 ? lanes_a : lanes_for(A.avg_row()), A, X, Z);
  dispatch_B<T, false>(s, b, lanes_at != 0 ? lanes_at : lanes_for(At.avg_row()), At, Z, Y);
}

template void csr_spmm<double>(cudaStream_t, const SparseView<double>&, int, const double*, double*, int);
template void csr_spmm<float>(cudaStream_t, const SparseView<float>&, int, const float*, float*, int);
template void ata_fused<double>(cudaStream_t, const SparseView<double>&, int, int, const double*, double*, int);
template void ata_fused<float>(cudaStream_t, const SparseView<float>&, int, int, const float*, float*, int);
template void ata_two_phase<double>(cudaStream_t, const SparseView<double>&, const SparseView<double>&, int,
                                    const double*, double*, double*, int, int);
template void ata_two_phase<float>(cudaStream_t, const SparseView<float>&, const SparseView<float>&, int,
                                   const float*, float*, float*, int, int);

// ---------------------------------------------------------------------------
// CSR -> CSC on the device: count, scan, scatter, then sort each column by row.
// ---------------------------------------------------------------------------
__global__ void k_count_cols(int64_t nnz, const int* __restrict__ ci, int* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[e]], 1);
}

// Exclusive scan of cnt[0..n) into out[0..n] by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_one_cta(int n, const int* __restrict__ cnt, int* __restrict__ out) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n ? cnt[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? warp_tot[w - 1] : 0);
    if (i < n) out[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

template <typename T>
__global__ void k_scatter_csc(int m, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ va,
                              const int* __restrict__ cp, int* __restrict__ fill, int* __restrict__ ri,
                              T* __restrict__ cv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int c = ci[e];
    const int pos = cp[c] + atomicAdd(&fill[c], 1);
    ri[pos] = i;
    cv[pos] = va[e];
  }
}

template <typename T>
__global__ void k_sort_cols(int n, const int* __restrict__ cp, int* __restrict__ ri, T* __restrict__ cv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int e0 = cp[c], e1 = cp[c + 1];
  for (int e = e0 + 1; e < e1; ++e) {  // insertion sort by row index (columns are short)
    const int r = ri[e];
    const T v = cv[e];
    int f = e - 1;
    while (f >= e0 && ri[f] > r) {
      ri[f + 1] = ri[f];
      cv[f + 1] = cv[f];
      --f;
    }
    ri[f + 1] = r;
    cv[f + 1] = v;
  }
}

template <typename T>
void csr_to_csc(cudaStream_t s, int m, int n, int64_t nnz, const int* rp, const int* ci, const T* va, int* cp,
                int* ri, T* cv, int* work_n) {
  cudaMemsetAsync(work_n, 0, sizeof(int) * (size_t)n, s);
  if (nnz > 0) k_count_cols<<<ceil_div(nnz, 256) < 4096 ? ceil_div(nnz, 256) : 4096, 256, 0, s>>>(nnz, ci, work_n); count_launch();
  k_scan_one_cta<<<1, 1024, 0, s>>>(n, work_n, cp); count_launch();
  cudaMemsetAsync(work_n, 0, sizeof(int) * (size_t)n, s);
  if (m > 0) k_scatter_csc<T><<<ceil_div(m, 256), 256, 0, s>>>(m, rp, ci, va, cp, work_n, ri, cv); count_launch();
  k_sort_cols<T><<<ceil_div(n, 256), 256, 0, s>>>(n, cp, ri, cv); count_launch();
}
template void csr_to_csc<double>(cudaStream_t, int, int, int64_t, const int*, const int*, const double*, int*, int*,
                                 double*, int*);

// FP64 CSR -> FP32 values (mixed precision copy of A).
__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
void to_float(cudaStream_t s, int64_t n, const double* a, float* b) {
  if (n > 0) k_to_float<<<ceil_div(n, 256) < 8192 ? ceil_div(n, 256) : 8192, 256, 0, s>>>(n, a, b); count_launch();
}

// diag(C)_j = sum_i a_ij^2 from the CSC copy (one thread per column).
__global__ void k_col_norms2(int n, const int* __restrict__ cp, const double* __restrict__ cv, double* __restrict__ d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double acc = 0.0;
  for (int e = cp[c]; e < cp[c + 1]; ++e) acc = fma(cv[e], cv[e], acc);
  d[c] = acc;
}
void col_norms2(cudaStream_t s, int n, const int* cp, const double* cv, double* d) {
  if (n > 0) k_col_norms2<<<ceil_div(n, 256), 256, 0, s>>>(n, cp, cv, d); count_launch();
}

// Validation of a CSR given with int64 row offsets, in two steps so that no
// kernel reads col/val through an unchecked offset:
//  1. k_rowptr_check: rp64[0] = 0, rp64[m] = nnz, non-decreasing, and converts
//     to int32 offsets clamped into [0, nnz] (flags |= 1 on violation);
//  2. k_validate_rows: indices in range and strictly increasing within a row
//     (flags |= 1), finite values (flags |= 2).
__global__ void k_rowptr_check(int m, int64_t nnz, const int64_t* __restrict__ rp64, int* __restrict__ rp32,
                               int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > m) return;
  const int64_t v = rp64[i];
  int bad = 0;
  if (v < 0 || v > nnz) bad = 1;
  if (i == 0 && v != 0) bad = 1;
  if (i == m && v != nnz) bad = 1;
  if (i < m && rp64[i + 1] < v) bad = 1;
  int64_t c = v < 0 ? 0 : (v > nnz ? nnz : v);
  rp32[i] = (int)c;
  if (bad) atomicOr(flags, 1);
}
__global__ void k_validate_rows(int m, int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ va, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int e0 = rp[i], e1 = rp[i + 1];
  int bad = 0;
  int prev = -1;
  for (int e = e0; e < e1; ++e) {
    const int c = ci[e];
    if (c < 0 || c >= n || c <= prev) { bad |= 1; break; }
    prev = c;
    if (!isfinite(va[e])) bad |= 2;
  }
  if (bad) atomicOr(flags, bad);
}
void rowptr_check(cudaStream_t s, int m, int64_t nnz, const int64_t* rp64, int* rp32, int* flags) {
  k_rowptr_check<<<ceil_div((int64_t)m + 1, 256), 256, 0, s>>>(m, nnz, rp64, rp32, flags); count_launch();
}
void validate_rows(cudaStream_t s, int m, int n, const int* rp, const int* ci, const double* va, int* flags) {
  if (m > 0) k_validate_rows<<<ceil_div(m, 256), 256, 0, s>>>(m, n, rp, ci, va, flags); count_launch();
}

}  // namespace ph
