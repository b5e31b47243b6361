// Deflated, Schwarz-preconditioned flexible GCR for D psi = eta (3.9).
//
// Paper: deflated equation (3.10)-(3.11), right preconditioning by M_sap
// (6.2), GCR with restarts and inexact preconditioning (Section 6.2),
// adapted little-solve precision and high-precision restart residuals (A.5).
//
// Every restart (mixed precision: D, Phi^+ and Phi in double-float arithmetic on FP64 fields, the
// little system by FP32 solves refined with FP64 residuals; plain: everything FP64):
//   rho = eta - D psi                            (rho = eta at the first restart, psi = 0)
//   c = A^{-1} Phi^+ rho  (little_tol_out); psi += Phi c; rho = eta - D psi
//   stop if ||rho|| <= tol ||eta||
//   one GCR cycle in the inner precision on  P_L D M_sap phi = rho / ||rho||:
//       xi_k = M_sap rho_k,  w = D xi_k,  chi_k = P_L w = w - D Phi A^{-1} Phi^+ w
//       (little tolerance min(cap, tol_in * ||rho_0|| / ||w||))
//       Gram-Schmidt of chi_k against chi_0..k-1, rho_{k+1} = rho_k - a_k chi_k
//   psi += ||rho|| * sum_k beta_k xi_k           FP64 accumulation
// The -Phi A^{-1} Phi^+ D zeta part of P_R zeta is supplied by the next
// restart's deflation correction, so psi ends as psi + P_R zeta + Phi A^{-1} Phi^+ rho.
// Several right-hand sides in mixed precision run the same algorithm in lockstep
// (solve_batch_f32): one batch through every kernel, converged right-hand sides frozen.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dw_common.cuh"

using cd = std::complex<double>;

// provided by dw_dfl.cu
int dfl_restrict_f32(dfl_ctx*, const float*, float*, cudaStream_t);
int dfl_restrict_f64(dfl_ctx*, const double*, double*, cudaStream_t);
int dfl_prolong_f32(dfl_ctx*, const float*, float*, int, cudaStream_t);
int dfl_prolong_f64(dfl_ctx*, const double*, double*, int, cudaStream_t);
int little_solve_f32(dfl_ctx*, const float*, float*, double, int, int, int*, double*, cudaStream_t);
int little_solve_f64(dfl_ctx*, const double*, double*, double, int, int, int*, double*, cudaStream_t);
int dfl_nlittle(const dfl_ctx*);
int dfl_restrict_mrhs_f32(dfl_ctx*, const float*, float*, int, cudaStream_t);
int dfl_prolong_mrhs_f32(dfl_ctx*, const float*, float*, int, int, cudaStream_t);
int little_solve_batch_f32(dfl_ctx*, const float*, float*, const double*, const int*, int, int, int, int*, double*,
                           cudaStream_t);
int little_solve_refined(dfl_ctx*, const double*, double*, double, int, int, int*, double*, cudaStream_t);
int dfl_restrict_f64x(dfl_ctx*, const double*, double*, cudaStream_t);
int little_solve_refined_batch(dfl_ctx*, const double*, double*, double, const int*, int, int, int, int*, double*,
                               cudaStream_t);
int dfl_prolong_f64x(dfl_ctx*, const double*, double*, int, cudaStream_t);

namespace {

inline int restrict_(dfl_ctx* d, const float* a, float* b, cudaStream_t s) { return dfl_restrict_f32(d, a, b, s); }
inline int restrict_(dfl_ctx* d, const double* a, double* b, cudaStream_t s) { return dfl_restrict_f64(d, a, b, s); }
inline int prolong_(dfl_ctx* d, const float* a, float* b, int m, cudaStream_t s) { return dfl_prolong_f32(d, a, b, m, s); }
inline int prolong_(dfl_ctx* d, const double* a, double* b, int m, cudaStream_t s) { return dfl_prolong_f64(d, a, b, m, s); }
inline int lsolve_(dfl_ctx* d, const float* w, float* v, double tol, int maxit, int nkv, int* it, double* rr,
                   cudaStream_t s) {
  return little_solve_f32(d, w, v, tol, maxit, nkv, it, rr, s);
}
inline int lsolve_(dfl_ctx* d, const double* w, double* v, double tol, int maxit, int nkv, int* it, double* rr,
                   cudaStream_t s) {
  return little_solve_f64(d, w, v, tol, maxit, nkv, it, rr, s);
}

enum Phase { PH_SAP, PH_DIRAC, PH_PROJECT, PH_LITTLE, PH_ORTH, PH_RESTART, PH_N };

struct Timers {
  cudaStream_t s;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PH_N];
  int open = -1;
  cudaEvent_t cur;
  void begin(int ph) {
    cudaEventCreate(&cur);
    cudaEventRecord(cur, s);
    open = ph;
  }
  void end() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev[open].push_back({cur, e});
    open = -1;
  }
  void collect(sol_info* in) {
    double t[PH_N] = {0};
    for (int p = 0; p < PH_N; ++p)
      for (auto& pr : ev[p]) {
        float ms = 0;
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        t[p] += ms * 1e-3;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
    if (in) {
      in->t_sap = t[PH_SAP]; in->t_dirac = t[PH_DIRAC]; in->t_project = t[PH_PROJECT];
      in->t_little = t[PH_LITTLE]; in->t_orth = t[PH_ORTH]; in->t_restart = t[PH_RESTART];
    }
  }
};

int read_host(dw_ctx* c, const double* dev, int n, double* host, cudaStream_t s) {
  DW_CUDA(cudaMemcpyAsync(c->h_red, dev, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) host[i] = c->h_red[i];
  return DW_OK;
}

// Views of a solver's fields in the context's workspace arena: the first solve of a shape
// allocates them, later solves of the same shape reuse them (no cudaMalloc/cudaFree per solve).
template <typename T>
struct Work {
  std::vector<T*> xi, chi;
  T *rho = nullptr, *w = nullptr, *t1 = nullptr, *lc = nullptr, *lv = nullptr;
  double *eta = nullptr, *psi = nullptr, *r64 = nullptr, *t64 = nullptr, *c64 = nullptr, *v64 = nullptr;
  dd *dda = nullptr, *ddb = nullptr;     // double-float fields of the mixed restarts
  WsArena& arena;
  explicit Work(WsArena& a) : arena(a) { arena.rewind(); }
  int alloc(size_t bytes, void** p) {
    cudaError_t e = arena.get(bytes, p);
    if (e != cudaSuccess) return dw_cuda_fail(e, "gcr_solve workspace");
    return DW_OK;
  }
};

template <typename T>
int solve_one(dw_ctx* c, dfl_ctx* d, const sol_params* p, const double* eta_canon, double* psi_canon,
              sol_info* info, cudaStream_t s) {
  constexpr int P = prec_of<T>();
  const size_t V = c->V;
  const size_t n = V * 12;              // complex numbers per field
  const size_t fbT = dw_field_bytes(c, P), fb64 = dw_field_bytes(c, DW_F64);
  const int nkv = p->nkv;
  const int Nl = d ? dfl_nlittle(d) : 0;
  Work<T> W(c->ws_solve[0]);
  int rc;
  W.xi.resize(nkv);
  W.chi.resize(nkv);
  for (int k = 0; k < nkv; ++k) {
    if ((rc = W.alloc(fbT, (void**)&W.xi[k])) || (rc = W.alloc(fbT, (void**)&W.chi[k]))) return rc;
  }
  if ((rc = W.alloc(fbT, (void**)&W.rho)) || (rc = W.alloc(fbT, (void**)&W.w)) || (rc = W.alloc(fbT, (void**)&W.t1)) ||
      (rc = W.alloc(fb64, (void**)&W.eta)) || (rc = W.alloc(fb64, (void**)&W.psi)) ||
      (rc = W.alloc(fb64, (void**)&W.r64)) || (rc = W.alloc(fb64, (void**)&W.t64)))
    return rc;
  if (d) {
    if ((rc = W.alloc((size_t)Nl * 2 * sizeof(T), (void**)&W.lc)) ||
        (rc = W.alloc((size_t)Nl * 2 * sizeof(T), (void**)&W.lv)) ||
        (rc = W.alloc((size_t)Nl * 2 * sizeof(double), (void**)&W.c64)) ||
        (rc = W.alloc((size_t)Nl * 2 * sizeof(double), (void**)&W.v64)))
      return rc;
  }
  Timers tm;
  tm.s = s;
  auto t_start = std::chrono::steady_clock::now();
  double* dres = c->d_red + 65536 + 4096;
  double h[2 * 64];
  if ((rc = dw_pack(c, DW_F64, 1, eta_canon, W.eta, s))) return rc;
  DW_CUDA(cudaMemsetAsync(W.psi, 0, fb64, s));
  blas_dot<double>(c, W.eta, W.eta, n, dres, s);
  if ((rc = read_host(c, dres, 3, h, s))) return rc;
  const double en = sqrt(h[2]);
  const bool verbose = getenv("DW_VERBOSE") && atoi(getenv("DW_VERBOSE")) > 0;
  sol_info inf{};
  inf.status = DW_ENOTCONV;
  if (en == 0.0) {
    inf.status = DW_OK;
    DW_CUDA(cudaMemsetAsync(psi_canon, 0, V * 24 * sizeof(double), s));
    if (info) *info = inf;
    return DW_OK;
  }
  if (p->mixed) {      // restart steps in double-float arithmetic on the FP32 pipes
    if ((rc = dw_make_dd(c, s)) || (rc = W.alloc(V * 24 * sizeof(dd), (void**)&W.dda)) ||
        (rc = W.alloc(V * 24 * sizeof(dd), (void**)&W.ddb)))
      return rc;
  }
  auto residual64 = [&]() -> int {   // r64 = eta - D psi, returns via h[2] = |r|^2
    tm.begin(PH_RESTART);
    if (p->mixed) {
      f64_to_dd(W.psi, W.dda, V * 24, s);
      dirac_full_dd(c, W.dda, W.ddb, s);
      dd_to_f64(W.ddb, W.t64, V * 24, 0, s);
    } else {
      dirac_full<double>(c, W.psi, W.t64, s);
    }
    DW_CUDA(cudaMemcpyAsync(W.r64, W.eta, fb64, cudaMemcpyDeviceToDevice, s));
    blas_axpy<double>(W.t64, W.r64, -1.0, 0.0, n, s);
    blas_dot<double>(c, W.r64, W.r64, n, dres, s);
    tm.end();
    return read_host(c, dres, 3, h, s);
  };
  std::vector<cd> a(nkv), cc(nkv), bb((size_t)nkv * nkv);
  double relres = 1.0;
  const int max_restarts = 10000;
  for (int restart = 0; restart < max_restarts; ++restart) {
    double rn;
    if (restart == 0) {     // psi = 0: the residual is eta
      DW_CUDA(cudaMemcpyAsync(W.r64, W.eta, fb64, cudaMemcpyDeviceToDevice, s));
      rn = en;
    } else {
      if ((rc = residual64())) return rc;
      rn = sqrt(h[2]);
    }
    if (d) {
      // deflation correction psi += Phi A^{-1} Phi^+ r in FP64 precision (A.5: high precision
      // outside the cycles; the error of the correction is amplified by the small eigenvalues
      // of A).  Mixed: FP32 little GCR with FP64 little residuals; else FP64 little GCR.
      int it = 0;
      double rr = 0;
      tm.begin(PH_PROJECT);
      if (p->mixed) rc = dfl_restrict_f64x(d, W.r64, W.c64, s);
      else restrict_(d, W.r64, W.c64, s);
      tm.end();
      if (rc < 0) return rc;
      tm.begin(PH_LITTLE);
      rc = p->mixed ? little_solve_refined(d, W.c64, W.v64, p->little_tol_out, p->little_maxit, p->little_nkv, &it,
                                           &rr, s)
                    : lsolve_(d, W.c64, W.v64, p->little_tol_out, p->little_maxit, p->little_nkv, &it, &rr, s);
      tm.end();
      if (rc < 0) return rc;
      tm.begin(PH_PROJECT);
      if (p->mixed) rc = dfl_prolong_f64x(d, W.v64, W.psi, 1, s);
      else prolong_(d, W.v64, W.psi, 1, s);
      tm.end();
      if (rc < 0) return rc;
      if ((rc = residual64())) return rc;
      rn = sqrt(h[2]);
      inf.little_iterations += it;
      inf.little_solves += 1;
    }
    relres = rn / en;
    if (verbose)
      fprintf(stderr, "[dwsolve] restart %d: |rho|/|eta| = %.3e  gcr steps %d  little its %d (%d solves)\n",
              restart, relres, inf.iterations, inf.little_iterations, inf.little_solves);
    if (rn <= p->tol * en) { inf.status = DW_OK; break; }
    if (inf.iterations >= p->nmx) break;
    // ---- one GCR cycle in precision T on rho / rn
    field_convert<double, T>(W.r64, W.rho, 1.0 / rn, V, s);
    const double stop = std::max(p->tol * en / rn, p->mixed ? p->inner_rtol : 0.0);
    int k = 0;
    double rk = 1.0;
    for (; k < nkv && inf.iterations < p->nmx; ++k) {
      tm.begin(PH_SAP);
      if (p->ncy > 0) {
        if ((rc = sap_apply<T>(c, p->ncy, p->nmr, W.rho, W.xi[k], s))) return rc;
      } else {   // no preconditioner (M = 1): plain GCR
        DW_CUDA(cudaMemcpyAsync(W.xi[k], W.rho, fbT, cudaMemcpyDeviceToDevice, s));
      }
      tm.end();
      tm.begin(PH_DIRAC);
      dirac_full<T>(c, W.xi[k], W.chi[k], s);
      tm.end();
      if (d) {
        // chi = P_L w = w - D Phi A^{-1} Phi^+ w, little tolerance adapted to |w| (A.5)
        tm.begin(PH_PROJECT);
        blas_dot<T>(c, W.chi[k], W.chi[k], n, dres, s);
        restrict_(d, W.chi[k], W.lc, s);
        tm.end();
        if ((rc = read_host(c, dres, 3, h, s))) return rc;
        double wn = sqrt(h[2]);
        double ltol = std::min(p->little_tol_cap, p->little_tol_in / std::max(wn, 1e-300));
        int it = 0;
        double rr = 0;
        tm.begin(PH_LITTLE);
        rc = lsolve_(d, W.lc, W.lv, ltol, p->little_maxit, p->little_nkv, &it, &rr, s);
        tm.end();
        if (rc < 0) return rc;
        inf.little_iterations += it;
        inf.little_solves += 1;
        tm.begin(PH_PROJECT);
        prolong_(d, W.lv, W.t1, 0, s);
        dirac_full<T>(c, W.t1, W.w, s);
        blas_axpy<T>(W.w, W.chi[k], -1.0, 0.0, n, s);
        tm.end();
      }
      tm.begin(PH_ORTH);
      if (k > 0) {
        std::vector<const T*> prev(W.chi.begin(), W.chi.begin() + k);
        blas_multi_dot<T>(c, prev.data(), k, W.chi[k], n, dres, s);
        if ((rc = read_host(c, dres, 2 * k, h, s))) return rc;
        for (int j = 0; j < k; ++j) bb[(size_t)j * nkv + k] = cd(h[2 * j], h[2 * j + 1]);
        blas_multi_axpy<T>(prev.data(), k, h, W.chi[k], n, s);
      }
      blas_dot<T>(c, W.chi[k], W.rho, n, dres, s);
      if ((rc = read_host(c, dres, 3, h, s))) return rc;
      double ck = sqrt(h[2]);
      if (!(ck > 0)) { tm.end(); break; }
      cc[k] = ck;
      a[k] = cd(h[0], h[1]) / ck;
      blas_scale<T>(W.chi[k], 1.0 / ck, 0.0, n, s);
      blas_axpy<T>(W.chi[k], W.rho, -a[k].real(), -a[k].imag(), n, s);
      blas_dot<T>(c, W.rho, W.rho, n, dres, s);
      if ((rc = read_host(c, dres, 3, h, s))) return rc;
      tm.end();
      rk = sqrt(h[2]);
      inf.iterations += 1;
      if (verbose > 0 && getenv("DW_VERBOSE")[0] == '2')
        fprintf(stderr, "[dwsolve]   step %d: |rho_k| = %.3e  c_k = %.3e\n", k, rk, ck);
      if (rk <= stop) { ++k; break; }
    }
    if (k == 0) break;
    std::vector<cd> beta(k);
    for (int j = k - 1; j >= 0; --j) {
      cd sacc = a[j];
      for (int i = j + 1; i < k; ++i) sacc -= bb[(size_t)j * nkv + i] * beta[i];
      beta[j] = sacc / cc[j];
    }
    std::vector<double> coef(2 * k);
    for (int j = 0; j < k; ++j) { coef[2 * j] = beta[j].real(); coef[2 * j + 1] = beta[j].imag(); }
    std::vector<const T*> xs(W.xi.begin(), W.xi.begin() + k);
    tm.begin(PH_RESTART);
    blas_lincomb<T>(xs.data(), k, coef.data(), W.w, n, s);
    field_convert<T, double>(W.w, W.t64, rn, V, s);
    blas_axpy<double>(W.t64, W.psi, 1.0, 0.0, n, s);
    tm.end();
    inf.restarts += 1;
  }
  if ((rc = dw_unpack(c, DW_F64, 1, W.psi, psi_canon, s))) return rc;
  DW_CUDA(cudaStreamSynchronize(s));
  inf.relres = relres;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  tm.collect(&inf);
  if (info) *info = inf;
  return inf.status;
}

// --------------------------------------------------------------------------- batched solve
// Mixed-precision DFL+SAP+GCR for nrhs right-hand sides in lockstep: every kernel processes the
// whole batch (links, clover and the deflation basis are read once per site or block for all
// right-hand sides), and each host round trip serves all of them.  A right-hand side that has
// converged is frozen (its psi is no longer updated).
int solve_batch_f32(dw_ctx* c, dfl_ctx* d, const sol_params* p, int nrhs, const double* eta_canon,
                    double* psi_canon, sol_info* info, cudaStream_t s) {
  const size_t V = c->V, n = V * 12, fs = V * 24;
  const size_t fb32 = dw_field_bytes(c, DW_F32) * nrhs, fb64 = dw_field_bytes(c, DW_F64) * nrhs;
  const int nkv = p->nkv;
  const int Nl = d ? dfl_nlittle(d) : 0;
  Work<float> W(c->ws_solve[1]);
  int rc;
  W.xi.resize(nkv);
  W.chi.resize(nkv);
  for (int k = 0; k < nkv; ++k)
    if ((rc = W.alloc(fb32, (void**)&W.xi[k])) || (rc = W.alloc(fb32, (void**)&W.chi[k]))) return rc;
  if ((rc = W.alloc(fb32, (void**)&W.rho)) || (rc = W.alloc(fb32, (void**)&W.w)) ||
      (rc = W.alloc(fb32, (void**)&W.t1)) || (rc = W.alloc(fb64, (void**)&W.eta)) ||
      (rc = W.alloc(fb64, (void**)&W.psi)) || (rc = W.alloc(fb64, (void**)&W.r64)) ||
      (rc = W.alloc(fb64, (void**)&W.t64)))
    return rc;
  if (d && ((rc = W.alloc((size_t)Nl * 2 * sizeof(float) * nrhs, (void**)&W.lc)) ||
            (rc = W.alloc((size_t)Nl * 2 * sizeof(float) * nrhs, (void**)&W.lv)) ||
            (rc = W.alloc((size_t)Nl * 2 * sizeof(double) * nrhs, (void**)&W.c64)) ||
            (rc = W.alloc((size_t)Nl * 2 * sizeof(double) * nrhs, (void**)&W.v64))))
    return rc;
  Timers tm;
  tm.s = s;
  auto t_start = std::chrono::steady_clock::now();
  double* dres = c->d_red + 65536 + 4096;
  std::vector<double> h(3 * 64 + 2 * 64 * 64);
  auto F32 = [&](float* base, int r) { return base + (size_t)r * fs; };
  auto F64 = [&](double* base, int r) { return base + (size_t)r * fs; };
  // batched norms / dots: one kernel per right-hand side, one read for all
  auto norms64 = [&](double* base, std::vector<double>& out) -> int {
    blas_dot_batch<double>(c, base, base, n, fs, nrhs, dres, s);
    int e = read_host(c, dres, 3 * nrhs, h.data(), s);
    for (int r = 0; r < nrhs; ++r) out[r] = sqrt(h[3 * r + 2]);
    return e;
  };
  if ((rc = dw_pack(c, DW_F64, nrhs, eta_canon, W.eta, s))) return rc;
  DW_CUDA(cudaMemsetAsync(W.psi, 0, fb64, s));
  std::vector<double> en(nrhs), rn(nrhs), relres(nrhs, 1.0), ltol(nrhs), rk(nrhs);
  std::vector<int> conv(nrhs, 0), live(nrhs), its(nrhs), lits(nrhs), nsteps(nrhs, 0), restarts(nrhs, 0),
      lsolves(nrhs, 0), litot(nrhs, 0);
  std::vector<double> lrr(nrhs);
  if ((rc = norms64(W.eta, en))) return rc;
  for (int r = 0; r < nrhs; ++r) conv[r] = en[r] == 0.0;
  dd *dda = nullptr, *ddb = nullptr;
  if ((rc = dw_make_dd(c, s)) || (rc = W.alloc(fs * sizeof(dd), (void**)&dda)) ||
      (rc = W.alloc(fs * sizeof(dd), (void**)&ddb)))
    return rc;
  auto residual64 = [&]() -> int {   // restart residuals in double-float arithmetic
    tm.begin(PH_RESTART);
    for (int r = 0; r < nrhs; ++r) {
      f64_to_dd(F64(W.psi, r), dda, fs, s);
      dirac_full_dd(c, dda, ddb, s);
      dd_to_f64(ddb, F64(W.t64, r), fs, 0, s);
    }
    DW_CUDA(cudaMemcpyAsync(W.r64, W.eta, fb64, cudaMemcpyDeviceToDevice, s));
    blas_axpy<double>(W.t64, W.r64, -1.0, 0.0, n * nrhs, s);   // the batch's fields are contiguous
    tm.end();
    return norms64(W.r64, rn);
  };
  const int nkvmax = nkv;
  std::vector<cd> a((size_t)nrhs * nkvmax), cc((size_t)nrhs * nkvmax), bb((size_t)nrhs * nkvmax * nkvmax);
  const int max_restarts = 10000;
  int total_steps = 0;
  for (int restart = 0; restart < max_restarts; ++restart) {
    if (restart == 0) {     // psi = 0: the residuals are the sources
      DW_CUDA(cudaMemcpyAsync(W.r64, W.eta, fb64, cudaMemcpyDeviceToDevice, s));
      rn = en;
    } else if ((rc = residual64())) {
      return rc;
    }
    if (d) {
      // deflation correction accurate to the outer tolerance (FP32 little iterations, FP64 residuals)
      tm.begin(PH_PROJECT);
      for (int r = 0; r < nrhs; ++r)
        if (!conv[r] && (rc = dfl_restrict_f64x(d, F64(W.r64, r), W.c64 + (size_t)r * Nl * 2, s))) return rc;
      tm.end();
      tm.begin(PH_LITTLE);
      {
        std::vector<int> use(nrhs), lit(nrhs);
        std::vector<double> lrr2(nrhs);
        for (int r = 0; r < nrhs; ++r) use[r] = !conv[r];
        rc = little_solve_refined_batch(d, W.c64, W.v64, p->little_tol_out, use.data(), p->little_maxit,
                                        p->little_nkv, nrhs, lit.data(), lrr2.data(), s);
        if (rc < 0) return rc;
        for (int r = 0; r < nrhs; ++r)
          if (use[r]) { litot[r] += lit[r]; lsolves[r] += 1; }
      }
      tm.end();
      tm.begin(PH_PROJECT);
      for (int r = 0; r < nrhs; ++r)
        if (!conv[r] && (rc = dfl_prolong_f64x(d, W.v64 + (size_t)r * Nl * 2, F64(W.psi, r), 1, s))) return rc;
      tm.end();
      if ((rc = residual64())) return rc;
    }
    bool all = true;
    for (int r = 0; r < nrhs; ++r) {
      if (!conv[r]) {
        relres[r] = rn[r] / en[r];
        if (rn[r] <= p->tol * en[r]) conv[r] = 1;
      }
      all &= conv[r] != 0;
    }
    if (all) break;
    if (total_steps >= p->nmx) break;
    // ---- one GCR cycle for the batch
    for (int r = 0; r < nrhs; ++r) {
      live[r] = !conv[r];
      field_convert<double, float>(F64(W.r64, r), F32(W.rho, r), live[r] ? 1.0 / rn[r] : 0.0, V, s);
      nsteps[r] = 0;
    }
    for (int k = 0; k < nkv && total_steps < p->nmx; ++k) {
      tm.begin(PH_SAP);
      if ((rc = sap_apply_mrhs_graph(c, p->ncy, p->nmr, W.rho, W.xi[k], nrhs, s))) return rc;
      tm.end();
      tm.begin(PH_DIRAC);
      dirac_mrhs<float>(c, W.xi[k], W.chi[k], nrhs, c->tune_rgroup, s);
      tm.end();
      if (d) {
        tm.begin(PH_PROJECT);
        blas_dot_batch<float>(c, W.chi[k], W.chi[k], n, fs, nrhs, dres, s);
        dfl_restrict_mrhs_f32(d, W.chi[k], W.lc, nrhs, s);
        tm.end();
        if ((rc = read_host(c, dres, 3 * nrhs, h.data(), s))) return rc;
        std::vector<int> use(nrhs);
        for (int r = 0; r < nrhs; ++r) {
          use[r] = live[r];
          ltol[r] = std::min(p->little_tol_cap, p->little_tol_in / std::max(sqrt(h[3 * r + 2]), 1e-300));
        }
        tm.begin(PH_LITTLE);
        rc = little_solve_batch_f32(d, W.lc, W.lv, ltol.data(), use.data(), p->little_maxit, p->little_nkv, nrhs,
                                    lits.data(), lrr.data(), s);
        tm.end();
        if (rc < 0) return rc;
        for (int r = 0; r < nrhs; ++r) if (use[r]) { litot[r] += lits[r]; lsolves[r] += 1; }
        tm.begin(PH_PROJECT);
        for (int r = 0; r < nrhs; ++r)
          if (!use[r]) DW_CUDA(cudaMemsetAsync(W.lv + (size_t)r * Nl * 2, 0, (size_t)Nl * 2 * sizeof(float), s));
        dfl_prolong_mrhs_f32(d, W.lv, W.t1, 0, nrhs, s);
        dirac_mrhs<float>(c, W.t1, W.w, nrhs, c->tune_rgroup, s);
        blas_axpy<float>(W.w, W.chi[k], -1.0, 0.0, n * nrhs, s);   // contiguous fields
        tm.end();
      }
      tm.begin(PH_ORTH);
      if (k > 0) {
        std::vector<const float*> prev0(k);
        for (int j = 0; j < k; ++j) prev0[j] = W.chi[j];
        const bool batched = nrhs <= 16;
        if (batched) {
          blas_multi_dot_batch<float>(c, prev0.data(), k, W.chi[k], n, fs, nrhs, dres, 2 * (size_t)nkv, s);
        } else {
          for (int r = 0; r < nrhs; ++r) {
            std::vector<const float*> prev(k);
            for (int j = 0; j < k; ++j) prev[j] = F32(W.chi[j], r);
            blas_multi_dot<float>(c, prev.data(), k, F32(W.chi[k], r), n, dres + (size_t)r * 2 * nkv, s);
          }
        }
        if ((rc = read_host(c, dres, 2 * nkv * nrhs, h.data(), s))) return rc;
        for (int r = 0; r < nrhs; ++r)
          for (int j = 0; j < k; ++j)
            bb[((size_t)r * nkvmax + j) * nkvmax + k] = cd(h[r * 2 * nkv + 2 * j], h[r * 2 * nkv + 2 * j + 1]);
        if (batched) {
          blas_multi_axpy_batch<float>(prev0.data(), k, h.data(), 2 * (size_t)nkv, W.chi[k], n, fs, nrhs, s);
        } else {
          for (int r = 0; r < nrhs; ++r) {
            std::vector<const float*> prev(k);
            for (int j = 0; j < k; ++j) prev[j] = F32(W.chi[j], r);
            blas_multi_axpy<float>(prev.data(), k, h.data() + (size_t)r * 2 * nkv, F32(W.chi[k], r), n, s);
          }
        }
      }
      blas_dot_batch<float>(c, W.chi[k], W.rho, n, fs, nrhs, dres, s);
      if ((rc = read_host(c, dres, 3 * nrhs, h.data(), s))) return rc;
      std::vector<double> sinv(nrhs, 0.0), sar(nrhs, 0.0), sai(nrhs, 0.0);
      for (int r = 0; r < nrhs; ++r) {
        double ck = sqrt(h[3 * r + 2]);
        if (!live[r] || !(ck > 0)) { live[r] = 0; continue; }
        cc[(size_t)r * nkvmax + k] = ck;
        a[(size_t)r * nkvmax + k] = cd(h[3 * r], h[3 * r + 1]) / ck;
        nsteps[r] = k + 1;
        sinv[r] = 1.0 / ck;
        sar[r] = a[(size_t)r * nkvmax + k].real();
        sai[r] = a[(size_t)r * nkvmax + k].imag();
      }
      // chi_k /= c_k, rho -= a_k chi_k and |rho|^2 for the live right-hand sides in one launch
      if (nrhs <= 16) {
        if ((rc = gcr_step_batch(c, W.chi[k], W.rho, n, fs, nrhs, sinv.data(), sar.data(), sai.data(), live.data(),
                                 dres, s)))
          return rc;
      } else {
        for (int r = 0; r < nrhs; ++r) {
          if (!live[r]) continue;
          blas_scale<float>(F32(W.chi[k], r), sinv[r], 0.0, n, s);
          blas_axpy<float>(F32(W.chi[k], r), F32(W.rho, r), -sar[r], -sai[r], n, s);
          blas_dot<float>(c, F32(W.rho, r), F32(W.rho, r), n, dres + 3 * r, s);
        }
      }
      if ((rc = read_host(c, dres, 3 * nrhs, h.data(), s))) return rc;
      tm.end();
      ++total_steps;
      bool any_live = false;
      for (int r = 0; r < nrhs; ++r) {
        if (!live[r]) continue;
        rk[r] = sqrt(h[3 * r + 2]);
        its[r] += 1;
        const double stop = std::max(p->tol * en[r] / rn[r], p->inner_rtol);
        if (rk[r] <= stop) live[r] = 0;     // this right-hand side's cycle is complete
        any_live |= live[r] != 0;
      }
      if (!any_live) break;
    }
    // psi += rn * sum_k beta_k xi_k  for every right-hand side with steps in this cycle
    tm.begin(PH_RESTART);
    for (int r = 0; r < nrhs; ++r) {
      const int kr = nsteps[r];
      if (conv[r] || kr == 0) continue;
      std::vector<cd> beta(kr);
      for (int j = kr - 1; j >= 0; --j) {
        cd sacc = a[(size_t)r * nkvmax + j];
        for (int i = j + 1; i < kr; ++i) sacc -= bb[((size_t)r * nkvmax + j) * nkvmax + i] * beta[i];
        beta[j] = sacc / cc[(size_t)r * nkvmax + j];
      }
      std::vector<double> coef(2 * kr);
      std::vector<const float*> xs(kr);
      for (int j = 0; j < kr; ++j) {
        coef[2 * j] = beta[j].real();
        coef[2 * j + 1] = beta[j].imag();
        xs[j] = F32(W.xi[j], r);
      }
      blas_lincomb<float>(xs.data(), kr, coef.data(), F32(W.w, r), n, s);
      field_convert<float, double>(F32(W.w, r), F64(W.t64, r), rn[r], V, s);
      blas_axpy<double>(F64(W.t64, r), F64(W.psi, r), 1.0, 0.0, n, s);
      restarts[r] += 1;
    }
    tm.end();
  }
  if ((rc = dw_unpack(c, DW_F64, nrhs, W.psi, psi_canon, s))) return rc;
  DW_CUDA(cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  sol_info agg{};
  tm.collect(&agg);
  int worst = DW_OK;
  for (int r = 0; r < nrhs; ++r) {
    sol_info in = agg;   // phase times are those of the whole batch
    in.status = conv[r] ? DW_OK : DW_ENOTCONV;
    in.iterations = its[r];
    in.restarts = restarts[r];
    in.little_iterations = litot[r];
    in.little_solves = lsolves[r];
    in.relres = relres[r];
    in.seconds = secs;
    if (info) info[r] = in;
    worst = std::max(worst, in.status);
  }
  return worst;
}

}  // namespace

extern "C" int gcr_solve(dw_ctx* c, dfl_ctx* d, const sol_params* p, int nrhs, const double* eta, double* psi,
                         sol_info* info, void* stream) {
  if (!c || !p || !eta || !psi || nrhs < 1 || p->nkv < 1 || p->nkv > 64 || p->nmx < 1 || !(p->tol > 0) ||
      p->ncy < 0 || p->nmr < 0 || (d && (p->little_nkv < 1 || p->little_maxit < 1))) {
    dw_set_error("gcr_solve: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "gcr_solve")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int worst = DW_OK;
  const size_t n = (size_t)c->V * 24;
  const char* be = getenv("DW_BATCH");
  if (p->mixed && nrhs > 1 && !(be && be[0] == '0') && p->nkv <= 64 && p->ncy > 0) {
    if (nrhs > 64) { dw_set_error("gcr_solve: at most 64 right-hand sides per batch"); return DW_EINVAL; }
    return solve_batch_f32(c, d, p, nrhs, eta, psi, info, s);
  }
  for (int r = 0; r < nrhs; ++r) {
    int rc = p->mixed ? solve_one<float>(c, d, p, eta + r * n, psi + r * n, info ? info + r : nullptr, s)
                      : solve_one<double>(c, d, p, eta + r * n, psi + r * n, info ? info + r : nullptr, s);
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
  }
  return worst;
}

// ------------------------------------------------------------------------- CGNR
// Conjugate gradient on the normal equations D^+ D psi = D^+ eta (CGLS form,
// recursively updated residual r = eta - D psi), FP64.  Used to measure the
// unpreconditioned CG iteration count that fixes the bare mass of a workload
// and as the plain comparison solver.  D^+ = gamma_5 D gamma_5; in the packed
// layout gamma_5 flips the sign of the second half of a field (spins 2, 3).
extern "C" int cgnr_solve(dw_ctx* c, double tol, int maxit, const double* eta_canon, double* psi_canon, int* iters,
                          double* relres, void* stream) {
  if (!c || !eta_canon || !psi_canon || maxit < 1 || !(tol > 0)) {
    dw_set_error("cgnr_solve: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "cgnr_solve")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t V = c->V, n = V * 12, fb = dw_field_bytes(c, DW_F64);
  Work<double> W(c->ws_solve[2]);
  double *b, *x, *r, *p, *q, *t;
  int rc;
  if ((rc = W.alloc(fb, (void**)&b)) || (rc = W.alloc(fb, (void**)&x)) || (rc = W.alloc(fb, (void**)&r)) ||
      (rc = W.alloc(fb, (void**)&p)) || (rc = W.alloc(fb, (void**)&q)) || (rc = W.alloc(fb, (void**)&t)))
    return rc;
  double* dres = c->d_red + 65536 + 8192;
  double h[3];
  auto gdag = [&](const double* in, double* out) -> int {   // out = gamma_5 D gamma_5 in
    DW_CUDA(cudaMemcpyAsync(t, in, fb, cudaMemcpyDeviceToDevice, s));
    blas_scale<double>(t + n, -1.0, 0.0, n / 2, s);
    dirac_full<double>(c, t, out, s);
    blas_scale<double>(out + n, -1.0, 0.0, n / 2, s);
    return DW_OK;
  };
  if ((rc = dw_pack(c, DW_F64, 1, eta_canon, b, s))) return rc;
  DW_CUDA(cudaMemsetAsync(x, 0, fb, s));
  DW_CUDA(cudaMemcpyAsync(r, b, fb, cudaMemcpyDeviceToDevice, s));
  blas_dot<double>(c, b, b, n, dres, s);
  if ((rc = read_host(c, dres, 3, h, s))) return rc;
  const double bn = sqrt(h[2]);
  if ((rc = gdag(r, p))) return rc;        // p = s = D^+ r
  blas_dot<double>(c, p, p, n, dres, s);
  if ((rc = read_host(c, dres, 3, h, s))) return rc;
  double gam = h[2], rn = bn;
  int it = 0;
  while (rn > tol * bn && it < maxit && gam > 0) {
    dirac_full<double>(c, p, q, s);
    blas_dot<double>(c, q, q, n, dres, s);
    if ((rc = read_host(c, dres, 3, h, s))) return rc;
    double alpha = gam / h[2];
    blas_axpy<double>(p, x, alpha, 0.0, n, s);
    blas_axpy<double>(q, r, -alpha, 0.0, n, s);
    if ((rc = gdag(r, q))) return rc;      // q = s = D^+ r
    blas_dot<double>(c, q, q, n, dres, s);
    double h2[3];
    if ((rc = read_host(c, dres, 3, h2, s))) return rc;
    blas_dot<double>(c, r, r, n, dres, s);
    if ((rc = read_host(c, dres, 3, h, s))) return rc;
    rn = sqrt(h[2]);
    double beta = h2[2] / gam;
    gam = h2[2];
    blas_xpby<double>(q, p, beta, 0.0, n, s);   // p = s + beta p
    ++it;
  }
  if ((rc = dw_unpack(c, DW_F64, 1, x, psi_canon, s))) return rc;
  DW_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = rn / bn;
  return rn <= tol * bn ? DW_OK : DW_ENOTCONV;
}

// ------------------------------------------------------------------------- EO+BiCGstab
// The first comparison solver of the paper's Table 1 (Section 6.3): BiCGstab on the even-odd
// preconditioned operator D^ = A_ee - D_eo A_oo^{-1} D_oe, FP64.  With psi_o reconstructed exactly,
// eta - D psi has no odd part and its even part is the residual of the even system, so the
// stopping rule ||eta - D psi|| <= tol ||eta|| is applied to ||b^ - D^ x|| (recursive residual,
// confirmed by the true residual with D; a confirmed miss restarts from the current x).
// iterations: BiCGstab iterations (two D^ applications each).
extern "C" int bicgstab_solve(dw_ctx* c, double tol, int maxit, const double* eta_canon, double* psi_canon,
                              int* iters, double* relres, void* stream) {
  if (!c || !eta_canon || !psi_canon || maxit < 1 || !(tol > 0)) {
    dw_set_error("bicgstab_solve: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "bicgstab_solve")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t V = c->V, n = V * 12, fb = dw_field_bytes(c, DW_F64);
  Work<double> W(c->ws_solve[2]);
  double *eta, *b, *x, *r, *r0, *p, *v, *sv, *t;
  int rc;
  if ((rc = W.alloc(fb, (void**)&eta)) || (rc = W.alloc(fb, (void**)&b)) || (rc = W.alloc(fb, (void**)&x)) ||
      (rc = W.alloc(fb, (void**)&r)) || (rc = W.alloc(fb, (void**)&r0)) || (rc = W.alloc(fb, (void**)&p)) ||
      (rc = W.alloc(fb, (void**)&v)) || (rc = W.alloc(fb, (void**)&sv)) || (rc = W.alloc(fb, (void**)&t)))
    return rc;
  double* dres = c->d_red + 65536 + 8192;
  double h[6];
  auto dot = [&](const double* a, const double* bb, double* out) -> int {   // out: Re, Im (a, bb), |a|^2
    blas_dot<double>(c, a, bb, n, dres, s);
    return read_host(c, dres, 3, out, s);
  };
  if ((rc = dw_pack(c, DW_F64, 1, eta_canon, eta, s))) return rc;
  if ((rc = dot(eta, eta, h))) return rc;
  const double en = sqrt(h[2]);
  DW_CUDA(cudaMemsetAsync(x, 0, fb, s));
  eo_prepare<double>(c, eta, b, t, s);
  int it = 0;
  double rn = en;
  bool done = en == 0.0;
  for (int attempt = 0; attempt < 4 && !done && it < maxit; ++attempt) {
    // r = b^ - D^ x, r0 = r
    if ((rc = dirac_schur<double>(c, x, t, s))) return rc;
    DW_CUDA(cudaMemcpyAsync(r, b, fb, cudaMemcpyDeviceToDevice, s));
    blas_axpy<double>(t, r, -1.0, 0.0, n, s);
    DW_CUDA(cudaMemcpyAsync(r0, r, fb, cudaMemcpyDeviceToDevice, s));
    DW_CUDA(cudaMemsetAsync(p, 0, fb, s));
    DW_CUDA(cudaMemsetAsync(v, 0, fb, s));
    cd rho = 1.0, alpha = 1.0, omega = 1.0;
    if ((rc = dot(r, r, h))) return rc;
    rn = sqrt(h[2]);
    while (rn > tol * en && it < maxit) {
      if ((rc = dot(r0, r, h))) return rc;
      const cd rho1(h[0], h[1]);
      if (std::abs(rho1) == 0.0 || std::abs(omega) == 0.0) break;          // breakdown: restart
      const cd beta = (rho1 / rho) * (alpha / omega);
      rho = rho1;
      // p = r + beta (p - omega v)
      blas_axpy<double>(v, p, -omega.real(), -omega.imag(), n, s);
      blas_xpby<double>(r, p, beta.real(), beta.imag(), n, s);
      if ((rc = dirac_schur<double>(c, p, v, s))) return rc;
      if ((rc = dot(r0, v, h))) return rc;
      const cd r0v(h[0], h[1]);
      if (std::abs(r0v) == 0.0) break;
      alpha = rho / r0v;
      // s = r - alpha v
      DW_CUDA(cudaMemcpyAsync(sv, r, fb, cudaMemcpyDeviceToDevice, s));
      blas_axpy<double>(v, sv, -alpha.real(), -alpha.imag(), n, s);
      if ((rc = dirac_schur<double>(c, sv, t, s))) return rc;
      if ((rc = dot(t, sv, h))) return rc;                // (t, s) and |t|^2
      if (!(h[2] > 0)) { blas_axpy<double>(p, x, alpha.real(), alpha.imag(), n, s); ++it; break; }
      omega = cd(h[0], h[1]) / h[2];
      // x += alpha p + omega s ; r = s - omega t
      blas_axpy<double>(p, x, alpha.real(), alpha.imag(), n, s);
      blas_axpy<double>(sv, x, omega.real(), omega.imag(), n, s);
      DW_CUDA(cudaMemcpyAsync(r, sv, fb, cudaMemcpyDeviceToDevice, s));
      blas_axpy<double>(t, r, -omega.real(), -omega.imag(), n, s);
      if ((rc = dot(r, r, h))) return rc;
      rn = sqrt(h[2]);
      ++it;
    }
    // true residual of the full system
    eo_reconstruct<double>(c, eta, x, sv, s);
    dirac_full<double>(c, sv, t, s);
    DW_CUDA(cudaMemcpyAsync(r, eta, fb, cudaMemcpyDeviceToDevice, s));
    blas_axpy<double>(t, r, -1.0, 0.0, n, s);
    if ((rc = dot(r, r, h))) return rc;
    rn = sqrt(h[2]);
    done = rn <= tol * en;
  }
  eo_reconstruct<double>(c, eta, x, sv, s);
  if ((rc = dw_unpack(c, DW_F64, 1, sv, psi_canon, s))) return rc;
  DW_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = en > 0 ? rn / en : 0.0;
  return rn <= tol * en ? DW_OK : DW_ENOTCONV;
}
