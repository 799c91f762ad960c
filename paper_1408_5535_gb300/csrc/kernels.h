// Internal declarations of the PHSVDS device kernels and their launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

struct phsvds_ctx;

namespace ph {

// Device and stream of a library handle (defined with the handle).
int handle_device(const phsvds_ctx* h);
cudaStream_t handle_stream(const phsvds_ctx* h);

// Runs f() once per CUDA device (the current one), safely from several host
// threads; used for per-function attributes such as the dynamic shared memory
// limit.  Two threads may both run f(): it must be idempotent.
template <typename F>
inline void once_per_device(std::atomic<uint64_t>& done, F&& f) {
  int d = 0;
  cudaGetDevice(&d);
  const uint64_t bit = 1ull << (d & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  f();
  done.fetch_or(bit, std::memory_order_acq_rel);
}

// A CSR view: nrows rows, ptr (nrows+1), idx, val (T).  The CSC copy of A is
// the CSR view of A^T.
template <typename T>
struct SparseView {
  int nrows = 0, ncols = 0;
  int64_t nnz = 0;
  const int* ptr = nullptr;
  const int* idx = nullptr;
  const T* val = nullptr;
  double avg_row() const { return nrows ? (double)nnz / nrows : 0.0; }
};

int lanes_for(double avg_row);

// Fixed-order reduction across thread blocks, so that repeated runs give the
// same bits: block b stores its partial results at ws + b * (n1 + n2), and a
// second launch (reduce_partials) adds them, in a fixed order, to
// out1[0 .. n1) and out2[0 .. n2).  With ws null the partials are added with
// atomics (order not fixed).  part: the block's partials in shared memory,
// complete when called; every thread calls.
struct RedWs {
  double* ws = nullptr;
};
__device__ inline void ordered_commit(const double* part, int n1, double* out1, int n2, double* out2, RedWs rw) {
  const int tid = threadIdx.x, nt = blockDim.x, no = n1 + n2;
  if (!rw.ws) {
    for (int o = tid; o < no; o += nt) atomicAdd(o < n1 ? &out1[o] : &out2[o - n1], part[o]);
    return;
  }
  double* mine = rw.ws + (size_t)blockIdx.x * no;
  for (int o = tid; o < no; o += nt) mine[o] = part[o];
}
// A block that has nothing to add still writes zeros to its slot (the second
// launch reads every slot); every thread calls.
__device__ inline void ordered_commit_zero(int no, RedWs rw) {
  if (!rw.ws) return;
  double* mine = rw.ws + (size_t)blockIdx.x * no;
  for (int o = threadIdx.x; o < no; o += blockDim.x) mine[o] = 0.0;
}
// The second half: out1/out2 += the partials of the `blocks` blocks, one warp
// per output (its lanes sum strided blocks, then a fixed butterfly), spread
// over as many SMs as there are outputs.  No-op when rw.ws is null.
void reduce_partials(cudaStream_t s, RedWs rw, int blocks, int n1, double* out1, int n2, double* out2);

// The host thread's scratch of the fixed-order cross-block reductions (set
// by a solve for its duration): {ws, counter} when it holds `doubles`, else
// {nullptr, nullptr} (the kernels then reduce with atomics).
RedWs red_ws(size_t doubles);
void set_red_ws(double* ws, size_t cap);

// Instrumentation (per host thread): kernel launch count, and optional CUDA
// events around kernel classes when a solve runs with opts.profile = 1.
// Classes 0-5 are the FP64 launches; 6-11 the same classes in FP32 storage.
enum ProfCat { PROF_CSPMM = 0, PROF_GRAM = 1, PROF_TALL = 2, PROF_SMALL = 3, PROF_SPMV = 4, PROF_JACOBI = 5, PROF_NCAT = 6,
               PROF_F32 = 6, PROF_NALL = 12 };
template <typename T> constexpr int pcat(int c) { return sizeof(T) == 4 ? c + PROF_F32 : c; }
void count_launch();
// Algorithmic work of a launch (per host thread, per kernel class): flops and
// the bytes the operation must move at least (each operand read once, each
// result written once), for the roofline of a profiled solve.
void count_work(int cat, double flops, double bytes);
void prof_begin(cudaStream_t s, int cat);
void prof_end(cudaStream_t s, int cat);
struct ProfScope {
  cudaStream_t s;
  int cat;
  ProfScope(cudaStream_t st, int c) : s(st), cat(c) { prof_begin(s, cat); }
  ~ProfScope() { prof_end(s, cat); }
};

// ---- sparse (k_sparse.cu)
// lanes: sparse-row group width (1, 2, 4, 8, 16); 0 picks it from the mean row
// length; -l: width l with 32-byte row gathers that do not allocate in L1.
template <typename T> void csr_spmm(cudaStream_t s, const SparseView<T>& A, int b, const T* X, T* Z, int lanes = 0);
template <typename T>
void ata_fused(cudaStream_t s, const SparseView<T>& A, int ncols, int b, const T* X, T* Y, int lanes = 0);
template <typename T>
void ata_two_phase(cudaStream_t s, const SparseView<T>& A, const SparseView<T>& At, int b, const T* X, T* Y, T* Z,
                   int lanes_a = 0, int lanes_at = 0);
template <typename T>
void csr_to_csc(cudaStream_t s, int m, int n, int64_t nnz, const int* rp, const int* ci, const T* va, int* cp,
                int* ri, T* cv, int* work_n);
void to_float(cudaStream_t s, int64_t n, const double* a, float* b);
void col_norms2(cudaStream_t s, int n, const int* cp, const double* cv, double* d);
void rowptr_check(cudaStream_t s, int m, int64_t nnz, const int64_t* rp64, int* rp32, int* flags);
void validate_rows(cudaStream_t s, int m, int n, const int* rp, const int* ci, const double* va, int* flags);

// ---- tall-skinny dense (k_tall.cu)
// All tall matrices are column-major with leading dimension ld (>= rows).
// A "Basis" is up to two column-major pieces [P1 | P2] seen as one.
template <typename T>
struct Basis {
  const T* p1 = nullptr; int ld1 = 0; int c1 = 0;
  const T* p2 = nullptr; int ld2 = 0; int c2 = 0;
  __host__ __device__ int cols() const { return c1 + c2; }
};

// One pass of block classical Gram-Schmidt over a block of q columns T
// (column-major, ld ldt):
//   if Gsub:  T <- T - P * Gsub      (Gsub: p x q, column-major ld p, FP64)
//   if Gout:  Gout += P^T T          (p x q, FP64, must be zeroed by caller)
//   if Tout:  Tout += T^T T          (q x q, FP64, must be zeroed by caller)
template <typename T>
void cgs_pass(cudaStream_t s, int n, const Basis<T>& P, T* Tb, int ldt, int q, const double* Gsub, double* Gout,
              double* Tout);

// Out (n x r, column-major ld ldo) = P (n x p) * Y (p x r, FP64 column-major ld ldy)
// [- Xs (n x r) * diag(theta)] when theta != nullptr.  In-place allowed when
// Out == P and r <= p (each thread reads its whole row before writing).
// If norms2 != nullptr: norms2[c] += ||Out(:,c)||^2 (FP64, zeroed by caller).
template <typename T>
void tall_times_small(cudaStream_t s, int n, const T* P, int ldp, int p, const double* Y, int ldy, int r, T* Out,
                      int ldo, const T* Xs, int ldx, const double* theta, double* norms2);

// T <- T * Linv^T  (q x q upper-triangular inverse factor applied on the right,
// FP64) and copy T into column-major destination Dst (ld ldd) when non-null.
template <typename T>
void scale_block(cudaStream_t s, int n, T* Tb, int ldt, int q, const double* M, T* Dst, int ldd);

// Column-major <-> row-major block copies (n x q).
template <typename T> void cm_to_rm(cudaStream_t s, int n, const T* src, int lds, int q, T* dst);
template <typename T> void rm_to_cm(cudaStream_t s, int n, const T* src, int q, T* dst, int ldd);

// Olsen/Jacobi correction: t_c = M r_c - e_c M x_c, M = diag(1/(d - theta_c)),
// e_c = (x^T M r)/(x^T M x); dots (2*q, FP64) computed by jacobi_dots first.
template <typename T>
void jacobi_dots(cudaStream_t s, int n, const double* d, const T* X, int ldx, const T* R, int ldr, int q,
                 const double* theta, double guard, double* dots);
template <typename T>
void jacobi_apply(cudaStream_t s, int n, const double* d, const T* X, int ldx, const T* R, int ldr, int q,
                  const double* theta, double guard, const double* dots, T* Tout, int ldt);

// Random uniform [-1,1) column (SplitMix64 stream) into column-major dst.
template <typename T> void fill_random(cudaStream_t s, int n, T* dst, uint64_t seed, uint64_t stream);
// dst = src (conversion between precisions).
void convert_f32_to_f64(cudaStream_t s, int64_t n, const float* a, double* b);
void convert_f64_to_f32(cudaStream_t s, int64_t n, const double* a, float* b);
// y = a*x + b*y on n doubles
void axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y);
// norms2[c] += ||X(:,c)||^2 for q columns (FP64 output)
template <typename T> void col_norms2_dense(cudaStream_t s, int n, const T* X, int ldx, int q, double* norms2);

void dot_accum(cudaStream_t s, int64_t n, const double* x, const double* y, double* out);
// y = x / d (|d| < guard raised to +-guard; guard 0: none)
void diag_div(cudaStream_t s, int64_t n, const double* x, const double* d, double guard, double* y);
// out = a - (dots[0] / dots[1]) b (a when dots[1] == 0): the Olsen combination
void olsen_combine(cudaStream_t s, int64_t n, const double* a, const double* b, const double* dots, double* out);
// y = x .* x
void square(cudaStream_t s, int64_t n, const double* x, double* y);
void scal(cudaStream_t s, int64_t n, double a, const double* ap, double* x);
template <typename T> void fill_const(cudaStream_t s, int64_t n, T v, T* x);

// ---- small one-CTA problems (k_small.cu), FP64, j <= 64
// Cyclic Jacobi on the symmetric j x j H (column-major, ld j); S <- S * J.
void jacobi_eig(cudaStream_t s, int j, double* H, double* S, double* theta, double tol, int max_sweeps,
                int* sweeps_out);
// One-sided Jacobi on G (j x j): G <- G J, S <- S J, sig = column norms of G.
void jacobi_svd(cudaStream_t s, int j, double* G, double* S, double* sig, double tol, int max_sweeps,
                int* sweeps_out);
// Cholesky of the q x q Gram P; writes Linv^T-style right factor M (q x q) with
// T * M orthonormal; flags[c] = 1 for columns whose pivot fell below
// drop^2 * max(P_cc, in_norm2[c]) (numerically dependent).
void chol_factor(cudaStream_t s, int q, const double* P, const double* in_norm2, double drop, double* M,
                 int* flags);
// C (r x c) = A^T (a x r)^T * B (a x c)   -- small dense product, FP64 column-major
void small_gemm_tn(cudaStream_t s, int a, int r, int c, const double* A, int lda, const double* B, int ldb,
                   double* C, int ldc);
void small_gemm_nn(cudaStream_t s, int r, int a, int c, const double* A, int lda, const double* B, int ldb,
                   double* C, int ldc);
// tol (times max |a_ij|) is the threshold of pairs touching one of the
// ntarget targets (smallest diagonal entries for tmode 0, largest for 1,
// closest to tshift for 2); the other pairs rotate when
// |a_pq| > tol_loose sqrt|a_pp a_qq| (relative); ntarget = 0 applies tol
// everywhere.  *sweeps_out = sweeps,
// *rot_out = rotations (either may be null).
void jacobi_eig_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                   int max_sweeps, int* sweeps_out, double tol_loose, int ntarget, int tmode, double tshift,
                   int* rot_out);
// Same as jacobi_eig_ld (FP64), spread over an 8-CTA thread-block cluster.
void jacobi_eig_cluster_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                           int max_sweeps, int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift,
                           int* rot_out);
// Same as jacobi_eig_ld in one CTA with the round's work compacted to the
// rotating pairs (shaped for GB300's narrow FP64 pipe).
void jacobi_eig_fast_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                        int max_sweeps, int* sweeps_out, double tol_rel, int ntarget, int tmode, double tshift,
                        int* rot_out);
// FP64 clean-up after an FP32 pass: Jacobi rotations of the pairs touching
// the ntarget targets only, to |a_tx| <= tol * max|a_ij|.
void jacobi_eig_targets_ld(cudaStream_t s, int j, double* H, int ldh, double* S, int lds, double* theta, double tol,
                           int max_sweeps, int* sweeps_out, int ntarget, int tmode, double tshift, int* rot_out);
// FP32 bulk pass: Sf (FP64 out) = the FP32 Jacobi rotation diagonalising H to
// ~tol * ||H||; H is not modified.
void jacobi_eig32_ld(cudaStream_t s, int j, const double* H, int ldh, double* Sf, int lds, double* theta, double tol,
                     int max_sweeps, int* sweeps_out, int* rot_out);
void jacobi_svd_ld(cudaStream_t s, int j, double* G, int ldg, double* S, int lds, double* sig, double tol,
                   int max_sweeps, int* sweeps_out);
void frame_append(cudaStream_t s, int j0, int nb, double* A, int lda, double* S, int lds, const double* Hn);
// order[0..j) = the indices of th by key: mode 0 ascending, 1 descending, 2
// by |th - shift|, 3 ascending among th > 1e-12 max |th| (the others last)
void order_theta(cudaStream_t s, int j, const double* th, int mode, double shift, int* order);
// bad (device int, may be null) is set when an index lies outside [0, j)
void gather_cols(cudaStream_t s, int j, const double* S, int lds, const int* idx, int nc, double* out, int ldo,
                 const double* th, double* th_out, int* bad = nullptr);
void build_transform(cudaStream_t s, int j, const double* S, int lds, const double* A, int lda, const double* cand,
                     int ldc, int nc, int nc_a, int lim_a, int a_orth, const double* excl, int lde, int ne, int nmax,
                     double* Y, int ldy, int* jn_out, double* A2, int lda2);
void set_identity(cudaStream_t s, int j, double* S, int lds);
void h_append(cudaStream_t s, int j0, int nb, double* H, int ldh, double* S, int lds, const double* Hn);
void ns_factor(cudaStream_t s, int j, double* F, int ldf);
void symmetrise(cudaStream_t s, int j, double* A, int lda);
void refined_inverse(cudaStream_t s, int j, const double* R, int ldr, const double* x0, const double* H, int ldh,
                     int maxit, double tau, double* s1_out, double* out, int* steps_out);
void qr_column(cudaStream_t s, int c, const double* g1, const double* g2, const double* tnorm2, double* R, int ldr,
               double* G, int ldg, double* SR, int ldsr, double* minv, int update_g);

// ---- conjugate gradients on (A^T A - shift I) x = r, up to 8 rhs in lockstep (k_tall.cu)
void cg_pq(cudaStream_t s, int n, int b, double shift, const double* P, double* Q, double* pq);
void cg_update(cudaStream_t s, int n, int b, const double* P, const double* Q, double* X, double* R,
               const double* rr, const double* pq, const int* act, double* rrn);
void cg_dir(cudaStream_t s, int n, int b, const double* R, double* P, const double* rr, const double* rrn,
            const int* act);
void cg_next(cudaStream_t s, int b, double* rr, double* rrn, const double* rr0, double tol2, double* pq, int* act,
             int* iters, int* bad);

// ---- inner solves of the Jacobi-Davidson correction equation (k_inner.cu)
// Vectors column-major n x q (q <= 8), FP32 or FP64.  acc: FP64 accumulators
// (32 + 8 nl doubles, zeroed by the caller before each reduction): [0,8)
// v^T C v, [8,16) v^T v, [16,24) x^T C v, [24,32) squared norms, [32, ...)
// Xl^T C v (nl x q, leading dimension nl).  sc: the MINRES scalars (17 x 8).
template <typename T> void jd_colnorms(cudaStream_t s, int n, int q, const T* R, double* acc);
template <typename T>
void jd_init(cudaStream_t s, int n, int q, const T* R, T* r1, T* r2, T* v, T* sol, T* w1, T* w2, const double* acc,
             double* sc);
template <typename T> void jd_dots(cudaStream_t s, int n, int q, const T* v, const T* X, const T* Cv, double* acc);
// One MINRES step.  u: the vector of the theta term (v itself, or in the
// scaled form the projected P D^{-1/2} v); ds: D^{-1/2} of the scaled form
// (null: none), applied to the operator's output before the recurrence; X null:
// no x term (the scaled form projects x as part of Xl).
template <typename T>
void jd_step(cudaStream_t s, int n, int q, int nl, const T* Cv, T* v, const T* u, const T* X, const T* Xl,
             const double* theta, const T* ds, T* r1, T* r2, T* w1, T* w2, T* sol, double* acc, double* sc,
             double tol);
// ds[i] = 1 / sqrt(max(d[i], guard)): D^{-1/2} for D = diag(C)
template <typename T> void jd_dscale(cudaStream_t s, int n, const double* d, double guard, T* ds);
// Y[:, c] = ds .* X[:, c] for the q columns (column-major, leading dimension n)
template <typename T> void jd_rowscale(cudaStream_t s, int n, int q, const T* ds, const T* X, T* Y);
// stage 2 (one FP64 system on B, dynamic stop by the eigen-residual of x + t):
// acc (256 doubles): [0] v^T Bv, [8] v^T v, [24] ||y||^2, [32, 32 + nq) Q^T Bv,
// [160, 163) the eigen-residual sums; sc: JD_NSCALAR * 8 + 8 doubles
void s2_start(cudaStream_t s, int64_t N, const double* R, double* r1, double* r2, double* v, double* t, double* w1,
              double* w2, double* Bt, double* Bw1, double* Bw2, double* acc, double* sc);
void s2_step(cudaStream_t s, int64_t N, int nq, const double* Bv, double* v, const double* Q, const double* mu,
             double* r1, double* r2, double* w1, double* w2, double* t, double* Bw1, double* Bw2, double* Bt,
             const double* x, const double* Bx, double* tbest, double* acc, double* sc, double eta_tol, int patience,
             int maxit);
constexpr int JD2_FIELD_STEPS = 17 * 8 + 5;   // sc index of the steps taken (stage-2 form)
constexpr int JD_NSCALAR = 17;
constexpr int JD_FIELD_ACT = 15;   // sc[JD_FIELD_ACT * 8 + c] != 0 while system c iterates

// ---- learned correction network (k_cnn.cu)
constexpr int CNN_NPARAM_H = 3024;
void cnn_weights(cudaStream_t s, const void* params_bf16, float* wf, float* wt);
void cnn_forward(cudaStream_t s, int B, int nx, int ny, const float* wf, const float* x, float* a1, float* a2,
                 float* y);
void cnn_backward(cudaStream_t s, int B, int nx, int ny, const float* wt, const float* x, const float* a1,
                  const float* a2, const float* y, const float* t, float* g3, float* g2, float* g1, double* tn2,
                  float* grad, double* loss);
void cnn_adam(cudaStream_t s, float* w, float* grad, float* m, float* v, int step, float lr, float b1, float b2,
              float eps, void* params_bf16);
template <typename T>
void cnn_pack(cudaStream_t s, int n, int nb, const T* R, int ldr, const double* norms2, const float* feat, float* x);
template <typename T> void cnn_unpack(cudaStream_t s, int n, int nb, const float* y, T* Tb, int ldt);

}  // namespace ph
