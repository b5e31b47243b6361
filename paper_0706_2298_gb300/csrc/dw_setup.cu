// Operator context: geometry tables, link import, clover term (Section 2.1
// operator: O(a)-improved Wilson with the clover-leaf field strength),
// packing between the canonical and the block-major layout.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include "dw_common.cuh"

// ------------------------------------------------------------------ errors
static thread_local std::string g_err = "no error";

void dw_set_error(const std::string& msg) { g_err = msg; }
int dw_check_device(const dw_ctx* c, const char* who) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dw_cuda_fail(e, who);
  if (dev != c->device) {
    char msg[200];
    snprintf(msg, sizeof msg, "%s: the current device (%d) is not the context's device (%d)", who, dev, c->device);
    dw_set_error(msg);
    return DW_EINVAL;
  }
  return DW_OK;
}
int dw_cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? DW_ENOMEM : DW_ECUDA;
}
extern "C" const char* dw_last_error(void) { return g_err.c_str(); }

static std::atomic<long long> g_launches{0};
void dw_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" long long dw_launch_count(void) { return g_launches.load(); }

// ------------------------------------------------------------------ clover kernel
// sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] restricted to the two chiral blocks,
// for the six planes mu < nu: sig[plane][block][a][b] (complex)
struct SigmaTable {
  double re[6][2][2][2];
  double im[6][2][2][2];
};

template <typename T>
__device__ void herm6_store(T* base, size_t V, size_t i, const cplx<double> (*A)[6]) {
  cplx<T> s[18];
  for (int j = 0; j < 3; ++j) s[j] = {(T)A[2 * j][2 * j].re, (T)A[2 * j + 1][2 * j + 1].re};
  int k = 3;
  for (int a = 0; a < 6; ++a)
    for (int b = a + 1; b < 6; ++b) s[k++] = {(T)A[a][b].re, (T)A[a][b].im};
  store_site<T, 18>(base, V, i, s);
}

// Gauss-Jordan inverse with partial pivoting; returns 0 on a zero pivot
__device__ int inv6(cplx<double> (*A)[6], cplx<double> (*X)[6]) {
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) X[a][b] = {a == b ? 1.0 : 0.0, 0.0};
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    double best = norm2(A[c][c]);
    for (int r = c + 1; r < 6; ++r)
      if (norm2(A[r][c]) > best) { best = norm2(A[r][c]); piv = r; }
    if (best == 0.0) return 0;
    if (piv != c)
      for (int b = 0; b < 6; ++b) {
        cplx<double> t = A[c][b]; A[c][b] = A[piv][b]; A[piv][b] = t;
        t = X[c][b]; X[c][b] = X[piv][b]; X[piv][b] = t;
      }
    cplx<double> p = A[c][c];
    double pn = norm2(p);
    cplx<double> pinv = {p.re / pn, -p.im / pn};
    for (int b = 0; b < 6; ++b) { A[c][b] = A[c][b] * pinv; X[c][b] = X[c][b] * pinv; }
    for (int r = 0; r < 6; ++r) {
      if (r == c) continue;
      cplx<double> f = A[r][c];
      for (int b = 0; b < 6; ++b) { A[r][b] -= f * A[c][b]; X[r][b] -= f * X[c][b]; }
    }
  }
  return 1;
}

__device__ void mat3_mul(const SU3<double>& A, const SU3<double>& B, SU3<double>& C) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) C.m[a][b] = A.m[a][0] * B.m[0][b] + A.m[a][1] * B.m[1][b] + A.m[a][2] * B.m[2][b];
}
__device__ void mat3_dag(const SU3<double>& A, SU3<double>& B) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) B.m[a][b] = conjg(A.m[b][a]);
}
__device__ void leaf(const SU3<double>& A, const SU3<double>& B, const SU3<double>& C, const SU3<double>& D,
                     SU3<double>& Q) {
  SU3<double> t1, t2;
  mat3_mul(A, B, t1);
  mat3_mul(t1, C, t2);
  mat3_mul(t2, D, t1);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Q.m[a][b] += t1.m[a][b];
}

__global__ void clover_build_kernel(Geom g, const double* __restrict__ links, SigmaTable sig, double diag,
                                    double csw, double* cl64, double* ci64, float* cl32, float* ci32,
                                    int* bad) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  size_t V = g.V;
  cplx<double> A[2][6][6];
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) A[k][a][b] = {a == b ? diag : 0.0, 0.0};
  int plane = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
      long long xpm = neighbour_of(g, i, 2 * mu), xmm = neighbour_of(g, i, 2 * mu + 1);
      long long xpn = neighbour_of(g, i, 2 * nu), xmn = neighbour_of(g, i, 2 * nu + 1);
      long long xmm_pn = neighbour_of(g, xmm, 2 * nu), xmm_mn = neighbour_of(g, xmm, 2 * nu + 1);
      long long xmn_pm = neighbour_of(g, xmn, 2 * mu);
      SU3<double> Um, Un, Um_pn, Un_pm, Um_mm, Un_mm, Um_mmpn, Un_mmmn, Um_mmmn, Un_mn, Um_mn, Un_mnpm;
      load_link(links, V, mu, i, Um);
      load_link(links, V, nu, i, Un);
      load_link(links, V, mu, xpn, Um_pn);
      load_link(links, V, nu, xpm, Un_pm);
      load_link(links, V, mu, xmm, Um_mm);
      load_link(links, V, nu, xmm, Un_mm);
      load_link(links, V, mu, xmm_pn, Um_mmpn);
      load_link(links, V, nu, xmm_mn, Un_mmmn);
      load_link(links, V, mu, xmm_mn, Um_mmmn);
      load_link(links, V, nu, xmn, Un_mn);
      load_link(links, V, mu, xmn, Um_mn);
      load_link(links, V, nu, xmn_pm, Un_mnpm);
      SU3<double> Q, d1, d2, d3, d4;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Q.m[a][b] = {0.0, 0.0};
      // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      mat3_dag(Um_pn, d1); mat3_dag(Un, d2);
      leaf(Um, Un_pm, d1, d2, Q);
      // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
      mat3_dag(Um_mmpn, d1); mat3_dag(Un_mm, d2);
      leaf(Un, d1, d2, Um_mm, Q);
      // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
      mat3_dag(Um_mm, d1); mat3_dag(Un_mmmn, d2);
      leaf(d1, d2, Um_mmmn, Un_mn, Q);
      // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
      mat3_dag(Un_mn, d3); mat3_dag(Um, d4);
      leaf(d3, Um_mn, Un_mnpm, d4, Q);
      // F = (Q - Q^+)/8 ; A_k += (i/2) csw sigma_k (x) F
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          cplx<double> F = 0.125 * (Q.m[c][d] - conjg(Q.m[d][c]));
          cplx<double> iF = {-0.5 * csw * F.im, 0.5 * csw * F.re};
          for (int k = 0; k < 2; ++k)
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) {
                cplx<double> s = {sig.re[plane][k][a][b], sig.im[plane][k][a][b]};
                A[k][3 * a + c][3 * b + d] += s * iF;
              }
        }
    }
  }
  for (int k = 0; k < 2; ++k) {
    herm6_store<double>(cl64 + 36 * V * k, V, i, A[k]);
    herm6_store<float>(cl32 + 36 * V * k, V, i, A[k]);
    cplx<double> X[6][6];
    if (!inv6(A[k], X)) { atomicExch(bad, 1); continue; }
    herm6_store<double>(ci64 + 36 * V * k, V, i, X);
    herm6_store<float>(ci32 + 36 * V * k, V, i, X);
  }
}

__global__ void pack_kernel64(const long long V, const int* __restrict__ canon_of, int nrhs,
                              const double* __restrict__ in, double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= V) return;
  long long x = canon_of[i];
  for (int r = 0; r < nrhs; ++r) {
    cplx<double> s[12];
    const double* src = in + (size_t)r * V * 24 + (size_t)x * 24;
    for (int k = 0; k < 12; ++k) s[k] = {src[2 * k], src[2 * k + 1]};
    store_site<double, 12>(out + (size_t)r * V * 24, V, i, s);
  }
}
__global__ void pack_kernel32(const long long V, const int* __restrict__ canon_of, int nrhs,
                              const double* __restrict__ in, float* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= V) return;
  long long x = canon_of[i];
  for (int r = 0; r < nrhs; ++r) {
    cplx<float> s[12];
    const double* src = in + (size_t)r * V * 24 + (size_t)x * 24;
    for (int k = 0; k < 12; ++k) s[k] = {(float)src[2 * k], (float)src[2 * k + 1]};
    store_site<float, 12>(out + (size_t)r * V * 24, V, i, s);
  }
}
template <typename T>
__global__ void unpack_kernel(const long long V, const int* __restrict__ canon_of, int nrhs,
                              const T* __restrict__ in, double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= V) return;
  long long x = canon_of[i];
  for (int r = 0; r < nrhs; ++r) {
    cplx<T> s[12];
    load_site<T, 12>(in + (size_t)r * V * 24, V, i, s);
    double* dst = out + (size_t)r * V * 24 + (size_t)x * 24;
    for (int k = 0; k < 12; ++k) { dst[2 * k] = (double)s[k].re; dst[2 * k + 1] = (double)s[k].im; }
  }
}

// ------------------------------------------------------------------ host helpers
static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

static void sigma_table(SigmaTable& t) {
  using C = std::complex<double>;
  const C I(0, 1);
  // e_0 = -1, e_k = -i sigma_k
  C e[4][2][2];
  const C vals[4][4] = {{C(-1), C(0), C(0), C(-1)},     // e_0 = -1
                        {C(0), -I, -I, C(0)},           // e_1 = -i sigma_1
                        {C(0), C(-1), C(1), C(0)},      // e_2 = -i sigma_2
                        {-I, C(0), C(0), I}};           // e_3 = -i sigma_3
  for (int m = 0; m < 4; ++m)
    for (int k = 0; k < 4; ++k) e[m][k / 2][k % 2] = vals[m][k];
  auto mul = [](const C (*a)[2], const C (*b)[2], C (*c)[2]) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) c[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j];
  };
  auto dag = [](const C (*a)[2], C (*b)[2]) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) b[i][j] = std::conj(a[j][i]);
  };
  int p = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++p) {
      C em_d[2][2], en_d[2][2], a[2][2], b[2][2];
      dag(e[mu], em_d);
      dag(e[nu], en_d);
      // gamma_mu gamma_nu = diag(e_mu e_nu^+, e_mu^+ e_nu)
      for (int k = 0; k < 2; ++k) {
        if (k == 0) { mul(e[mu], en_d, a); mul(e[nu], em_d, b); }
        else        { mul(em_d, e[nu], a); mul(en_d, e[mu], b); }
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) {
            C s = 0.5 * I * (a[i][j] - b[i][j]);
            t.re[p][k][i][j] = s.real();
            t.im[p][k][i][j] = s.imag();
          }
      }
    }
}

static void put_cplx(std::vector<char>& buf, int prec, size_t V, size_t field_off_reals, size_t i, int k,
                     double re, double im) {
  int CU = prec == DW_F64 ? 1 : 2;
  size_t u = k / CU, w = k % CU;
  size_t off = field_off_reals + u * (2 * CU) * V + i * (2 * CU) + w * 2;
  if (prec == DW_F64) {
    double* d = reinterpret_cast<double*>(buf.data());
    d[off] = re; d[off + 1] = im;
  } else {
    float* f = reinterpret_cast<float*>(buf.data());
    f[off] = (float)re; f[off + 1] = (float)im;
  }
}

static void free_ctx(dw_ctx* c) {
  if (!c) return;
  sap_graphs_free(c);
  for (auto& a : c->ws_solve) a.release();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* ptrs[] = {c->d_canon_of, c->d_nbtab, c->d_blk_nb, c->d_blk_x0, c->d_loc, c->d_colour_list,
                  c->links[0], c->links[1], c->clov[0], c->clov[1], c->clovinv[0], c->clovinv[1],
                  c->sap_r[0], c->sap_r[1], c->sap_d[0], c->sap_d[1], c->d_red, c->d_count,
                  c->links_dd, c->clov_dd};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_red) cudaFreeHost(c->h_red);
  delete c;
}

extern "C" void dw_destroy(dw_ctx* c) { free_ctx(c); }

extern "C" int dw_release_workspace(dw_ctx* c) {
  if (!c) { dw_set_error("dw_release_workspace: null context"); return DW_EINVAL; }
  if (int rc = dw_check_device(c, "dw_release_workspace")) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return dw_cuda_fail(e, "dw_release_workspace");
  for (auto& a : c->ws_solve) a.release();
  if (c->links_dd) { cudaFree(c->links_dd); c->links_dd = nullptr; }
  if (c->clov_dd) { cudaFree(c->clov_dd); c->clov_dd = nullptr; }
  return DW_OK;
}

extern "C" size_t dw_field_bytes(const dw_ctx* c, int prec) {
  return c ? (size_t)c->V * 24 * real_size(prec) : 0;
}
extern "C" long long dw_volume(const dw_ctx* c) { return c ? c->V : 0; }

extern "C" int dw_create(const dw_params* p, const double* links_host, dw_ctx** out) {
  if (!p || !links_host || !out) { dw_set_error("dw_create: null argument"); return DW_EINVAL; }
  *out = nullptr;
  long long V = 1;
  int nsb[4];
  for (int mu = 0; mu < 4; ++mu) {
    int L = p->L[mu], b = p->sap_bs[mu];
    if (L <= 0 || b < 2 || !is_pow2(b) || L % b != 0 || (L / b) % 2 != 0) {
      dw_set_error("dw_create: each sap_bs[mu] must be a power of two >= 2 dividing L[mu] an even number of times");
      return DW_EINVAL;
    }
    nsb[mu] = L / b;
    V *= L;
  }
  int svol = p->sap_bs[0] * p->sap_bs[1] * p->sap_bs[2] * p->sap_bs[3];
  if (svol > 512) { dw_set_error("dw_create: Schwarz blocks are limited to 512 sites"); return DW_EINVAL; }
  if (V > (1LL << 31) - 1) { dw_set_error("dw_create: lattice too large"); return DW_EINVAL; }

  // SU(3) check on the host (canonical layout)
  for (long long x = 0; x < V * 4; ++x) {
    const double* u = links_host + x * 18;
    std::complex<double> U[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) U[a][b] = {u[2 * (3 * a + b)], u[2 * (3 * a + b) + 1]};
    double dev = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        std::complex<double> s = 0;
        for (int k = 0; k < 3; ++k) s += U[a][k] * std::conj(U[b][k]);
        dev = std::max(dev, std::abs(s - (a == b ? 1.0 : 0.0)));
      }
    std::complex<double> det = U[0][0] * (U[1][1] * U[2][2] - U[1][2] * U[2][1]) -
                               U[0][1] * (U[1][0] * U[2][2] - U[1][2] * U[2][0]) +
                               U[0][2] * (U[1][0] * U[2][1] - U[1][1] * U[2][0]);
    dev = std::max(dev, std::abs(det - 1.0));
    if (!(dev <= 1e-10)) {
      char msg[160];
      snprintf(msg, sizeof msg, "dw_create: link %lld (site %lld, mu %lld) is not SU(3) (deviation %.3g)", x,
               x / 4, x % 4, dev);
      dw_set_error(msg);
      return DW_EINVAL;
    }
  }

  int dev = -1;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dw_cuda_fail(e, "dw_create: cudaGetDevice");
  }
  dw_ctx* c = new dw_ctx();
  c->p = *p;
  c->device = dev;
  {
    uint64_t h = 1469598103934665603ull;       // FNV-1a over the bytes of the canonical links
    const unsigned char* b = reinterpret_cast<const unsigned char*>(links_host);
    const size_t nb = (size_t)V * 4 * 18 * sizeof(double);
    for (size_t k = 0; k < nb; ++k) { h ^= b[k]; h *= 1099511628211ull; }
    c->gauge_hash = h;
  }
  c->V = V;
  for (int mu = 0; mu < 4; ++mu) c->nsb[mu] = nsb[mu];
  Geom& g = c->g;
  for (int mu = 0; mu < 4; ++mu) { g.L[mu] = p->L[mu]; g.sb[mu] = p->sap_bs[mu]; }
  g.V = V;
  g.svol = svol;
  g.shv = svol / 2;
  g.lsvol = ilog2(svol);
  g.lshv = ilog2(svol / 2);
  g.nsap = nsb[0] * nsb[1] * nsb[2] * nsb[3];
  g.antiperiodic = p->antiperiodic ? 1 : 0;
  const int* sb = p->sap_bs;
  const int* L = p->L;

  // block tables
  std::vector<int> blk_nb((size_t)g.nsap * 8), blk_x0(g.nsap), bcoord((size_t)g.nsap * 4);
  c->blk_colour.resize(g.nsap);
  for (int b = 0; b < g.nsap; ++b) {
    int r = b, bc[4];
    for (int mu = 3; mu >= 0; --mu) { bc[mu] = r % nsb[mu]; r /= nsb[mu]; }
    for (int mu = 0; mu < 4; ++mu) bcoord[b * 4 + mu] = bc[mu];
    blk_x0[b] = bc[0] * sb[0];
    c->blk_colour[b] = (bc[0] + bc[1] + bc[2] + bc[3]) & 1;
    for (int d = 0; d < 8; ++d) {
      int mu = d / 2, s = (d & 1) ? -1 : 1;
      int nc[4] = {bc[0], bc[1], bc[2], bc[3]};
      nc[mu] = (nc[mu] + s + nsb[mu]) % nsb[mu];
      blk_nb[b * 8 + d] = ((nc[0] * nsb[1] + nc[1]) * nsb[2] + nc[2]) * nsb[3] + nc[3];
    }
  }
  // local tables
  int shv = g.shv;
  std::vector<uchar4> loc(2 * shv);
  std::vector<uint16_t> nbtab((size_t)2 * shv * 8);
  auto local_lex = [&](const int* l) { return ((l[0] * sb[1] + l[1]) * sb[2] + l[2]) * sb[3] + l[3]; };
  for (int par = 0; par < 2; ++par)
    for (int h = 0; h < shv; ++h) {
      int lx = 2 * h, l[4];
      l[3] = lx % sb[3]; lx /= sb[3];
      l[2] = lx % sb[2]; lx /= sb[2];
      l[1] = lx % sb[1]; l[0] = lx / sb[1];
      l[3] += (par + l[0] + l[1] + l[2]) & 1;
      loc[par * shv + h] = make_uchar4(l[0], l[1], l[2], l[3]);
      for (int d = 0; d < 8; ++d) {
        int mu = d / 2, s = (d & 1) ? -1 : 1;
        int n[4] = {l[0], l[1], l[2], l[3]};
        n[mu] += s;
        int cross = 0;
        if (n[mu] < 0) { n[mu] += sb[mu]; cross = 1; }
        if (n[mu] >= sb[mu]) { n[mu] -= sb[mu]; cross = 1; }
        nbtab[((size_t)par * shv + h) * 8 + d] = (uint16_t)((local_lex(n) >> 1) | (cross << 15));
      }
    }
  // internal -> canonical
  c->canon_of.resize(V);
  for (int b = 0; b < g.nsap; ++b)
    for (int par = 0; par < 2; ++par)
      for (int h = 0; h < shv; ++h) {
        uchar4 l = loc[par * shv + h];
        int x[4] = {bcoord[b * 4 + 0] * sb[0] + l.x, bcoord[b * 4 + 1] * sb[1] + l.y,
                    bcoord[b * 4 + 2] * sb[2] + l.z, bcoord[b * 4 + 3] * sb[3] + l.w};
        long long ci = ((x[0] * (long long)L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3];
        c->canon_of[(size_t)b * svol + par * shv + h] = (int)ci;
      }
  std::vector<int> colour_list;
  for (int col = 0; col < 2; ++col) {
    for (int b = 0; b < g.nsap; ++b)
      if (c->blk_colour[b] == col) colour_list.push_back(b);
    c->ncolour[col] = (int)colour_list.size() - (col ? c->ncolour[0] : 0);
  }

  // links in the packed layout (rows 0 and 1)
  std::vector<char> l64((size_t)V * 4 * 12 * 8), l32((size_t)V * 4 * 12 * 4);
  for (long long i = 0; i < V; ++i) {
    long long x = c->canon_of[i];
    for (int mu = 0; mu < 4; ++mu) {
      const double* u = links_host + (x * 4 + mu) * 18;
      for (int k = 0; k < 6; ++k) {
        put_cplx(l64, DW_F64, V, (size_t)mu * 12 * V, i, k, u[2 * k], u[2 * k + 1]);
        put_cplx(l32, DW_F32, V, (size_t)mu * 12 * V, i, k, u[2 * k], u[2 * k + 1]);
      }
    }
  }

  int rc = DW_OK;
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return dw_cuda_fail(e, "cudaMalloc");
    if (src) {
      e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return dw_cuda_fail(e, "cudaMemcpy");
    }
    return DW_OK;
  };
  if ((rc = up((void**)&c->d_canon_of, c->canon_of.data(), V * sizeof(int))) ||
      (rc = up((void**)&c->d_nbtab, nbtab.data(), nbtab.size() * sizeof(uint16_t))) ||
      (rc = up((void**)&c->d_blk_nb, blk_nb.data(), blk_nb.size() * sizeof(int))) ||
      (rc = up((void**)&c->d_blk_x0, blk_x0.data(), blk_x0.size() * sizeof(int))) ||
      (rc = up((void**)&c->d_loc, loc.data(), loc.size() * sizeof(uchar4))) ||
      (rc = up((void**)&c->d_colour_list, colour_list.data(), colour_list.size() * sizeof(int))) ||
      (rc = up(&c->links[DW_F64], l64.data(), l64.size())) ||
      (rc = up(&c->links[DW_F32], l32.data(), l32.size())) ||
      (rc = up(&c->clov[DW_F64], nullptr, (size_t)V * 72 * 8)) ||
      (rc = up(&c->clov[DW_F32], nullptr, (size_t)V * 72 * 4)) ||
      (rc = up(&c->clovinv[DW_F64], nullptr, (size_t)V * 72 * 8)) ||
      (rc = up(&c->clovinv[DW_F32], nullptr, (size_t)V * 72 * 4)) ||
      (rc = up((void**)&c->d_red, nullptr, 1 << 20)) ||
      (rc = up((void**)&c->d_count, nullptr, 64 * sizeof(unsigned)))) {
    free_ctx(c);
    return rc;
  }
  cudaMemset(c->d_count, 0, 64 * sizeof(unsigned));
  if (cudaMallocHost((void**)&c->h_red, 1 << 16) != cudaSuccess) {
    free_ctx(c);
    dw_set_error("dw_create: pinned allocation failed");
    return DW_ENOMEM;
  }
  g.nbtab = c->d_nbtab;
  g.blk_nb = c->d_blk_nb;
  g.blk_x0 = c->d_blk_x0;
  g.loc = c->d_loc;

  // clover term and its inverse (FP64 build, FP32 copies)
  SigmaTable sig;
  sigma_table(sig);
  int* d_bad = (int*)(c->d_count + 32);
  int threads = 128;
  long long blocks = (V + threads - 1) / threads;
  clover_build_kernel<<<(unsigned)blocks, threads>>>(g, (const double*)c->links[DW_F64], sig, 4.0 + p->m0, p->csw,
                                                     (double*)c->clov[DW_F64], (double*)c->clovinv[DW_F64],
                                                     (float*)c->clov[DW_F32], (float*)c->clovinv[DW_F32], d_bad); dw_note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { rc = dw_cuda_fail(e, "clover_build_kernel"); free_ctx(c); return rc; }
  if (bad) { dw_set_error("dw_create: singular clover block"); free_ctx(c); return DW_EINVAL; }
  cudaMemset(d_bad, 0, sizeof(int));
  *out = c;
  return DW_OK;
}

extern "C" int dw_pack(dw_ctx* c, int prec, int nrhs, const double* in, void* out, void* stream) {
  if (!c || !in || !out || nrhs < 1 || (prec != DW_F64 && prec != DW_F32)) {
    dw_set_error("dw_pack: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned blocks = (unsigned)((c->V + 127) / 128);
  if (prec == DW_F64) { pack_kernel64<<<blocks, 128, 0, s>>>(c->V, c->d_canon_of, nrhs, in, (double*)out); dw_note_launch(); }
  else { pack_kernel32<<<blocks, 128, 0, s>>>(c->V, c->d_canon_of, nrhs, in, (float*)out); dw_note_launch(); }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

extern "C" int dw_unpack(dw_ctx* c, int prec, int nrhs, const void* in, double* out, void* stream) {
  if (!c || !in || !out || nrhs < 1 || (prec != DW_F64 && prec != DW_F32)) {
    dw_set_error("dw_unpack: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned blocks = (unsigned)((c->V + 127) / 128);
  if (prec == DW_F64) { unpack_kernel<double><<<blocks, 128, 0, s>>>(c->V, c->d_canon_of, nrhs, (const double*)in, out); dw_note_launch(); }
  else { unpack_kernel<float><<<blocks, 128, 0, s>>>(c->V, c->d_canon_of, nrhs, (const float*)in, out); dw_note_launch(); }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
