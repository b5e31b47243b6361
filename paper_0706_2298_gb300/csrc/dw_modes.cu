// Low modes of D^+ D and the local-coherence deficits.
//
// The paper computes all eigenvalues and eigenmodes of D^+ D with Chebyshev-accelerated subspace
// iteration (Section 2.2) and measures local coherence (Section 5.2) by building a domain-decomposed
// subspace (4.1)-(4.2) from some of the low modes and evaluating the deficits (3.15) of the others.
//
// Subspace iteration (Rutishauser; the filtered block is re-orthonormalised and Rayleigh-Ritz
// projected every iteration):
//   Y <- T_deg(L(A)) Y,  L(A) = (2 A - (b + a)) / (b - a),  A = D^+ D  (b >= lambda_max(A),
//        a = largest Ritz value of the block: the Chebyshev polynomial is bounded by 1 on [a, b]
//        and grows fast below a, so the low end of the spectrum is amplified)
//   Y <- orthonormal basis of Y (classical Gram-Schmidt, two passes, FP64)
//   H = Y^+ A Y,  H = V diag(theta) V^+,  Y <- Y V  (Ritz vectors, ascending theta)
//   stop when ||A y_i - theta_i y_i|| <= tol theta_i for the nev lowest.
// The filter runs in FP32 or FP64 (multi-RHS D over the whole block), the Rayleigh-Ritz step in FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <type_traits>
#include <vector>

#include "dw_common.cuh"

using cd = std::complex<double>;

int dfl_restrict_f64(dfl_ctx*, const double*, double*, cudaStream_t);
int dfl_prolong_f64(dfl_ctx*, const double*, double*, int, cudaStream_t);
int dfl_nlittle(const dfl_ctx*);
dw_ctx* dfl_operator(const dfl_ctx*);

namespace {

int read_dev(dw_ctx* c, const double* dev, size_t n, double* host, cudaStream_t s) {
  DW_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  return DW_OK;
}

// out = gamma_5 D gamma_5 D in for nrhs packed fields (tmp: nrhs fields).  In the packed layout
// gamma_5 flips the sign of the second half of a field (spins 2 and 3).
template <typename T>
void ddag_d(dw_ctx* c, const T* in, T* out, T* tmp, int nrhs, cudaStream_t s) {
  const size_t fs = (size_t)c->V * 24, half = fs / 2;
  if (nrhs == 1) dirac_full<T>(c, in, tmp, s); else dirac_mrhs<T>(c, in, tmp, nrhs, c->tune_rgroup, s);
  for (int r = 0; r < nrhs; ++r) blas_scale<T>(tmp + r * fs + half, -1.0, 0.0, half / 2, s);
  if (nrhs == 1) dirac_full<T>(c, tmp, out, s); else dirac_mrhs<T>(c, tmp, out, nrhs, c->tune_rgroup, s);
  for (int r = 0; r < nrhs; ++r) blas_scale<T>(out + r * fs + half, -1.0, 0.0, half / 2, s);
}

// H = V diag(w) V^+ for a Hermitian n x n matrix (row-major), cyclic Jacobi rotations; w ascending,
// V's columns the eigenvectors.  In the (p, q) plane the rotation diagonalises
// [[a, h], [conj(h), b]] = D [[a, r], [r, b]] D^+ with h = r e^{i phi}, D = diag(1, e^{-i phi}):
// U = D R with the real Jacobi rotation R = [[c, s], [-s, c]].
void herm_eig(int n, std::vector<cd> H, std::vector<double>& w, std::vector<cd>& V) {
  V.assign((size_t)n * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, diag = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += std::norm(H[(size_t)i * n + j]);
    if (off <= 1e-30 * std::max(diag, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd h = H[(size_t)p * n + q];
        const double r = std::abs(h);
        if (r <= 1e-300) continue;
        const cd e = h / r;                                // e^{i phi}
        const double a = H[(size_t)p * n + p].real(), b = H[(size_t)q * n + q].real();
        const double zeta = (b - a) / (2 * r);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(zeta * zeta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        const cd em = std::conj(e);                        // e^{-i phi}
        // columns: M = H U   (U_pp = c, U_pq = s, U_qp = -s e^{-i phi}, U_qq = c e^{-i phi})
        for (int k = 0; k < n; ++k) {
          const cd hp = H[(size_t)k * n + p], hq = H[(size_t)k * n + q];
          H[(size_t)k * n + p] = cs * hp - sn * em * hq;
          H[(size_t)k * n + q] = sn * hp + cs * em * hq;
          const cd vp = V[(size_t)k * n + p], vq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = cs * vp - sn * em * vq;
          V[(size_t)k * n + q] = sn * vp + cs * em * vq;
        }
        // rows: H = U^+ M   (U^+_pp = c, U^+_pq = -s e^{i phi}, U^+_qp = s, U^+_qq = c e^{i phi})
        for (int k = 0; k < n; ++k) {
          const cd mp = H[(size_t)p * n + k], mq = H[(size_t)q * n + k];
          H[(size_t)p * n + k] = cs * mp - sn * e * mq;
          H[(size_t)q * n + k] = sn * mp + cs * e * mq;
        }
        H[(size_t)p * n + q] = 0.0;
        H[(size_t)q * n + p] = 0.0;
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return H[(size_t)x * n + x].real() < H[(size_t)y * n + y].real(); });
  std::vector<cd> Vs((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = H[(size_t)idx[j] * n + idx[j]].real();
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + j] = V[(size_t)k * n + idx[j]];
  }
  V.swap(Vs);
}

// Gram-Schmidt of the n packed FP64 fields Y (classical, two passes): orthonormal columns
int orthonormalise(dw_ctx* c, std::vector<double*>& Y, double* dres, cudaStream_t s) {
  const size_t nc = (size_t)c->V * 12;
  const int n = (int)Y.size();
  std::vector<double> h(2 * (size_t)n + 3);
  for (int j = 0; j < n; ++j) {
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      std::vector<const double*> prev(Y.begin(), Y.begin() + j);
      blas_multi_dot<double>(c, prev.data(), j, Y[j], nc, dres, s);
      if (int rc = read_dev(c, dres, 2 * (size_t)j, h.data(), s)) return rc;
      blas_multi_axpy<double>(prev.data(), j, h.data(), Y[j], nc, s);
    }
    blas_dot<double>(c, Y[j], Y[j], nc, dres, s);
    if (int rc = read_dev(c, dres, 3, h.data(), s)) return rc;
    if (!(h[2] > 0)) { dw_set_error("lowmodes_solve: the block lost rank"); return DW_EINVAL; }
    blas_scale<double>(Y[j], 1.0 / std::sqrt(h[2]), 0.0, nc, s);
  }
  return DW_OK;
}

}  // namespace

extern "C" int lowmodes_solve(dw_ctx* c, int nev, int nbuf, int degree, double tol, int maxit, int prec,
                              const double* start, double* modes, double* evals, double* resid, int* iters,
                              void* stream) {
  if (!c || !start || !modes || !evals || nev < 1 || nbuf < 0 || nev + nbuf > 128 || degree < 1 || !(tol > 0) ||
      maxit < 1 || (prec != DW_F32 && prec != DW_F64)) {
    dw_set_error("lowmodes_solve: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "lowmodes_solve")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = nev + nbuf;
  const size_t V = c->V, fs = V * 24, nc = V * 12;
  const size_t fb64 = fs * sizeof(double), fbp = fs * sizeof(double);   // filter blocks sized for FP64
  WsArena& ar = c->ws_solve[3];
  ar.rewind();
  double *Yb, *Wb, *Xb, *tmp, *dres;
  void *f0, *f1, *ft;
  cudaError_t ae = cudaSuccess;
  for (auto pr : {std::make_pair(fb64 * n, (void**)&Yb), std::make_pair(fb64 * n, (void**)&Wb),
                  std::make_pair(fb64 * n, (void**)&Xb), std::make_pair(fb64, (void**)&tmp),
                  std::make_pair(fbp * n, &f0), std::make_pair(fbp * n, &f1), std::make_pair(fbp * n, &ft),
                  std::make_pair(sizeof(double) * (2 * (size_t)n * n + 64), (void**)&dres)})
    if (ae == cudaSuccess) ae = ar.get(pr.first, pr.second);
  if (ae != cudaSuccess) return dw_cuda_fail(ae, "lowmodes_solve workspace");
  int rc;
  auto col = [&](double* base, int j) { return base + (size_t)j * fs; };
  if ((rc = dw_pack(c, DW_F64, n, start, Yb, s))) return rc;
  // upper bound of the spectrum of A: power iteration on the first start field, 1.1 x the estimate
  double bmax = 0;
  {
    std::vector<double> h(3);
    DW_CUDA(cudaMemcpyAsync(Xb, Yb, fb64, cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < 40; ++it) {
      blas_dot<double>(c, Xb, Xb, nc, dres, s);
      if ((rc = read_dev(c, dres, 3, h.data(), s))) return rc;
      blas_scale<double>(Xb, 1.0 / std::sqrt(h[2]), 0.0, nc, s);
      ddag_d<double>(c, Xb, Wb, tmp, 1, s);
      blas_dot<double>(c, Xb, Wb, nc, dres, s);           // Rayleigh quotient of the unit vector
      if ((rc = read_dev(c, dres, 3, h.data(), s))) return rc;
      bmax = std::max(bmax, h[0]);
      DW_CUDA(cudaMemcpyAsync(Xb, Wb, fb64, cudaMemcpyDeviceToDevice, s));
    }
    bmax *= 1.1;
  }
  std::vector<double*> Y(n), X(n), W(n);
  for (int j = 0; j < n; ++j) { Y[j] = col(Yb, j); X[j] = col(Xb, j); W[j] = col(Wb, j); }
  std::vector<double> theta(n, 0.0), res(n, 0.0), h(2 * (size_t)n * n + 8);
  std::vector<cd> H((size_t)n * n), Vm;
  double a_cut = 0;
  int it = 0, nconv = 0;
  int fprec = prec;                 // filter precision: an FP32 filter hands over to FP64 when it stalls
  double last = INFINITY;
  for (; it <= maxit; ++it) {
    if (it > 0) {
      // Chebyshev filter of the block: y_{k+1} = 2 L(A) y_k - y_{k-1}, y_1 = L(A) y_0
      const double al = 2.0 / (bmax - a_cut), be = -(bmax + a_cut) / (bmax - a_cut);
      auto filter = [&](auto* t0, auto* t1, auto* tt) {
        using T = std::remove_pointer_t<decltype(t0)>;
        const size_t ntot = nc * n;
        for (int j = 0; j < n; ++j) field_convert<double, T>(Y[j], t0 + (size_t)j * fs, 1.0, V, s);
        ddag_d<T>(c, t0, t1, tt, n, s);                     // t1 = A y0
        blas_scale<T>(t1, al, 0.0, ntot, s);
        blas_axpy<T>(t0, t1, be, 0.0, ntot, s);             // t1 = L y0
        T* ym = t0;
        T* yc = t1;
        for (int k = 2; k <= degree; ++k) {
          ddag_d<T>(c, yc, tt, reinterpret_cast<T*>(Xb), n, s);   // tt = A y_k  (Xb as scratch)
          blas_scale<T>(ym, -1.0, 0.0, ntot, s);
          blas_axpy<T>(tt, ym, 2 * al, 0.0, ntot, s);
          blas_axpy<T>(yc, ym, 2 * be, 0.0, ntot, s);       // ym = 2 L y_k - y_{k-1}
          std::swap(ym, yc);
        }
        for (int j = 0; j < n; ++j) field_convert<T, double>(yc + (size_t)j * fs, Y[j], 1.0, V, s);
      };
      if (fprec == DW_F32) filter((float*)f0, (float*)f1, (float*)ft);
      else filter((double*)f0, (double*)f1, (double*)ft);
    }
    if ((rc = orthonormalise(c, Y, dres, s))) return rc;
    // Rayleigh-Ritz: W = A Y, H = Y^+ W
    ddag_d<double>(c, Yb, Wb, Xb, n, s);
    for (int j = 0; j < n; ++j) {
      std::vector<const double*> ys(Y.begin(), Y.end());
      blas_multi_dot<double>(c, ys.data(), n, W[j], nc, dres + 2 * (size_t)j * n, s);
    }
    if ((rc = read_dev(c, dres, 2 * (size_t)n * n, h.data(), s))) return rc;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const cd hij(h[2 * ((size_t)j * n + i)], h[2 * ((size_t)j * n + i) + 1]);   // (y_i, A y_j)
        const cd hji(h[2 * ((size_t)i * n + j)], h[2 * ((size_t)i * n + j) + 1]);
        H[(size_t)i * n + j] = 0.5 * (hij + std::conj(hji));
      }
    herm_eig(n, H, theta, Vm);
    // Ritz vectors X = Y V and their residuals |A x_i - theta_i x_i| = |W v_i - theta_i x_i|
    std::vector<double> coef(2 * (size_t)n);
    std::vector<const double*> ys(Y.begin(), Y.end()), ws(W.begin(), W.end());
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        coef[2 * j] = Vm[(size_t)j * n + i].real();
        coef[2 * j + 1] = Vm[(size_t)j * n + i].imag();
      }
      blas_lincomb<double>(ys.data(), n, coef.data(), X[i], nc, s);
      if (i < nev) {
        blas_lincomb<double>(ws.data(), n, coef.data(), tmp, nc, s);
        blas_axpy<double>(X[i], tmp, -theta[i], 0.0, nc, s);
        blas_dot<double>(c, tmp, tmp, nc, dres + 2 * (size_t)n * n + 3 * 0, s);
        if ((rc = read_dev(c, dres + 2 * (size_t)n * n, 3, h.data(), s))) return rc;
        res[i] = std::sqrt(h[2]);
      }
    }
    std::swap(Yb, Xb);
    for (int j = 0; j < n; ++j) { Y[j] = col(Yb, j); X[j] = col(Xb, j); }
    nconv = 0;
    while (nconv < nev && res[nconv] <= tol * std::max(theta[nconv], 1e-300)) ++nconv;
    a_cut = theta[n - 1];
    if (nconv == nev) break;
    // the rounding of an FP32 filter limits the residuals to about 1e-7 lambda_max: once the first
    // unconverged residual no longer halves per iteration, the filter continues in FP64
    const double cur = res[nconv] / std::max(theta[nconv], 1e-300);
    if (fprec == DW_F32 && it >= 2 && cur > 0.5 * last) fprec = DW_F64;
    last = cur;
  }
  if ((rc = dw_unpack(c, DW_F64, nev, Yb, modes, s))) return rc;
  DW_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < nev; ++i) {
    evals[i] = theta[i];
    if (resid) resid[i] = res[i];
  }
  if (iters) *iters = std::min(it, maxit);
  return nconv == nev ? DW_OK : DW_ENOTCONV;
}

// eps_f = ||(1 - P) psi_f||^2 / ||psi_f||^2 with P the block projector (4.1) of the subspace
extern "C" int dfl_deficits(dfl_ctx* d, int nf, const double* fields, double* eps, void* stream) {
  if (!d || nf < 1 || !fields || !eps) { dw_set_error("dfl_deficits: bad argument"); return DW_EINVAL; }
  dw_ctx* c = dfl_operator(d);
  if (int rc = dw_check_device(c, "dfl_deficits")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t V = c->V, fs = V * 24, nc = V * 12;
  const size_t Nl = (size_t)dfl_nlittle(d);
  double *x, *px, *cl, *dres;
  DW_CUDA(cudaMallocAsync((void**)&x, fs * sizeof(double), s));
  DW_CUDA(cudaMallocAsync((void**)&px, fs * sizeof(double), s));
  DW_CUDA(cudaMallocAsync((void**)&cl, Nl * 2 * sizeof(double), s));
  DW_CUDA(cudaMallocAsync((void**)&dres, 8 * sizeof(double), s));
  int rc = DW_OK;
  double h[6];
  for (int f = 0; f < nf && rc == DW_OK; ++f) {
    if ((rc = dw_pack(c, DW_F64, 1, fields + f * fs, x, s))) break;
    if ((rc = dfl_restrict_f64(d, x, cl, s)) < 0) break;
    if ((rc = dfl_prolong_f64(d, cl, px, 0, s)) < 0) break;
    rc = DW_OK;
    blas_dot<double>(c, x, x, nc, dres, s);
    blas_axpy<double>(x, px, -1.0, 0.0, nc, s);                 // px = P x - x
    blas_dot<double>(c, px, px, nc, dres + 3, s);
    if ((rc = read_dev(c, dres, 6, h, s))) break;
    eps[f] = h[2] > 0 ? h[5] / h[2] : 0.0;
  }
  cudaFreeAsync(x, s);
  cudaFreeAsync(px, s);
  cudaFreeAsync(cl, s);
  cudaFreeAsync(dres, s);
  if (rc == DW_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dw_cuda_fail(e, "dfl_deficits");
  }
  return rc;
}
