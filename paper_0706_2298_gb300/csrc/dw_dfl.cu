// Deflation subspace and little Dirac operator.
//
//   Section 4.1  block projection  P psi = sum_L sum_l phi^L_l (phi^L_l, psi)
//   Section 4.2  phi^L_l = Gram-Schmidt of psi_l restricted to block L
//   Section 5.3  inverse iteration psi_l <- "D^{-1}" psi_l with M_sap  (5.1)
//   (3.2), A.1   B_{LL'} = (phi^L_k, D phi^{L'}_l)  (L' = L or one of 8 neighbours)
//   A.2          even-odd little operator  B^ = 1 - B_ee^{-1} B_eo B_oo^{-1} B_oe
//   A.3          global-mode deflation of the little system
//   A.4          GCR on the deflated even-odd little system: one persistent cooperative kernel
//                per solve (FP32 or FP64), and a multi-RHS variant that solves up to 12
//                systems in lockstep (FP32, batched right-hand sides)
//   A.5          FP64-accurate restart solves by iterative refinement (FP32 solves, FP64
//                residuals), single and batched
//
// Restriction and prolongation run in FP32, FP64 or double-float arithmetic (FP64 fields on the
// FP32 pipes, for the restart steps of the mixed solver).
//
// Basis storage: Ns global fields (field l = sum_L phi^L_l) in the packed
// layout; FP64 for the plain path, BF16 (3 x 16-byte units of 4 complex per
// site) for the mixed path.  The FP64 copy always holds the values the
// little operator is built from (dequantised when BF16 is stored).
// Little vectors: complex[Nb][Ns], block = lexicographic deflation-block index.
#include <chrono>
#include <cmath>
#include <complex>
#include <cooperative_groups.h>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "dw_common.cuh"

namespace cg = cooperative_groups;

extern "C" int ptnet_forward(dw_ctx* c, int C, const void* W, int nf, const void* x, void* y, void* stream);

using cd = std::complex<double>;

struct dfl_ctx {
  dw_ctx* c = nullptr;
  dfl_params p{};
  int bs[4], nb[4];
  int Nb = 0, Ns = 0, N = 0, nsub = 0;
  int* d_sub = nullptr;        // [Nb][nsub] Schwarz blocks of each deflation block
  int* d_sap2dfl = nullptr;    // [nsap]
  int* d_bnb = nullptr;        // [Nb][8] neighbouring deflation block
  // parity lists
  int Ne = 0, No = 0;
  int* d_list[2] = {nullptr, nullptr};   // block ids of parity 0 / 1
  int* d_lnb[2] = {nullptr, nullptr};    // [n_par][8] position of the neighbour in the other list
  // basis
  double* basis64 = nullptr;
  uint4* basis16 = nullptr;
  // little operator
  double* B64 = nullptr;                 // [Nb][9][Ns][Ns] column-major complex
  float* B32 = nullptr;                  // FP32 copy
  void* fw[2] = {nullptr, nullptr};      // full-system fallback work (A.2)
  double* Binv64 = nullptr; float* Binv32 = nullptr;   // [Nb][Ns][Ns]
  double* M64 = nullptr; float* M32 = nullptr;         // [Nb][8][Ns][Ns]  B_LL^{-1} B_{L,nb(L,d)}
  bool illcond = false;
  double max_cond = 0;
  // global-mode deflation (A.3)
  bool a3 = false;
  double* g64 = nullptr; float* g32 = nullptr;         // [Ns][Ne*Ns]
  double* Bg64 = nullptr; float* Bg32 = nullptr;       // B^ g
  std::vector<cd> Atil_inv;                            // Ns x Ns row-major
  std::vector<int> hlist0;                             // even blocks (host copy of d_list[0])
  std::vector<cd> graw;                                // [Ns][Ne*Ns] (phi^L_k, psi_l) on even blocks (A.3 input)
  double* Ainv64 = nullptr; float* Ainv32 = nullptr;   // device copies of A~^{-1}
  int coop_grid = 0;                                   // CTAs of the cooperative little solver (0: not possible)
  bool coop_m = false;                                 // multi-RHS cooperative little solver available
  float* mw = nullptr;                                 // its work: 2 COOP_NKV + 6 vectors of COOP_MRP systems
  float* mio = nullptr;                                // right-hand sides and solutions [2][COOP_MAXR][Ne Ns]
  float* meo = nullptr;                                // odd-part work [2][COOP_MAXR][No Ns]
  double* macc = nullptr;                              // reduction accumulators [3][COOP_MNV]
  float* mscr = nullptr;                               // per-CTA coefficient tables of the multi-RHS solver
  float* mtol = nullptr;                               // tolerances [COOP_MAXR]
  double* mout = nullptr;                              // iterations, relative residuals [COOP_MAXR][2]
  int defer_slot = -1;                                 // >= 0: write results to coop_out[2*slot], no host sync
  double* ref64 = nullptr;                             // refinement work: 3 FP64 little vectors
  float* ref32 = nullptr;                              //                  2 FP32 little vectors
  double* coop_partial = nullptr;                      // reduction accumulators of the cooperative solver
  double* coop_out = nullptr;                          // iterations, relative residual
  int* coop_err = nullptr;                             // error flag of the ring variant
  bool coop_ring = false;                              // FP32 cooperative solver with the shared-memory ring
  dd* ddf = nullptr;                                   // double-float field (restriction/prolongation)
  dd* ddl = nullptr;                                   // double-float little vector
  // work vectors (little GCR)
  void* lw[2] = {nullptr, nullptr};                    // per precision
  size_t lw_count = 0;
};

namespace {

constexpr int NSMAX = 32;

// ------------------------------------------------------------------ BF16 basis units
DW_D void bf16_unpack4(const uint4& u, cplx<float>* c) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 f = __bfloat1622float2(h[j]);
    c[j] = {f.x, f.y};
  }
}
template <typename T>
DW_D void load_basis(const double* b64, const uint4* b16, size_t V, int l, size_t i, cplx<T>* out) {
  if (b16) {
    const uint4* p = b16 + (size_t)l * 3 * V;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      cplx<float> c[4];
      bf16_unpack4(__ldg(p + (size_t)u * V + i), c);
#pragma unroll
      for (int j = 0; j < 4; ++j) out[4 * u + j] = {(T)c[j].re, (T)c[j].im};
    }
  } else {
    cplx<double> c[12];
    load_site<double, 12>(b64 + (size_t)l * 24 * V, V, i, c);
#pragma unroll
    for (int j = 0; j < 12; ++j) out[j] = {(T)c[j].re, (T)c[j].im};
  }
}

template <typename T>
DW_D T block_sum(T v, T* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T s = 0;
  for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += sh[j];
  return s;
}

// iterate over the sites of deflation block L: site index of the t-th site
DW_D long long dfl_site(const Geom& g, const int* sub, int nsub, int L, int t) {
  int sb = sub[L * nsub + (t >> g.lsvol)];
  return ((long long)sb << g.lsvol) + (t & (g.svol - 1));
}

// ------------------------------------------------------------------ Gram-Schmidt (FP64)
__global__ void __launch_bounds__(256) block_gs_kernel(Geom g, const int* __restrict__ sub, int nsub, int Ns,
                                                       double* basis, int* rank_loss) {
  __shared__ double sh[8];
  const int L = blockIdx.x;
  const size_t V = g.V;
  const int nsite = nsub * g.svol;
  for (int l = 0; l < Ns; ++l) {
    double* vl = basis + (size_t)l * 24 * V;
    double n0 = 0;
    for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
      cplx<double> a[12];
      load_site_rw<double, 12>(vl, V, dfl_site(g, sub, nsub, L, t), a);
      for (int k = 0; k < 12; ++k) n0 += norm2(a[k]);
    }
    n0 = sqrt(block_sum(n0, sh));
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < l; ++j) {
        const double* vj = basis + (size_t)j * 24 * V;
        double cr = 0, ci = 0;
        for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
          long long i = dfl_site(g, sub, nsub, L, t);
          cplx<double> a[12], b[12];
          load_site_rw<double, 12>(vj, V, i, a);
          load_site_rw<double, 12>(vl, V, i, b);
          for (int k = 0; k < 12; ++k) {
            cplx<double> z = cmulc(a[k], b[k]);
            cr += z.re; ci += z.im;
          }
        }
        cr = block_sum(cr, sh);
        ci = block_sum(ci, sh);
        cplx<double> cc = {cr, ci};
        for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
          long long i = dfl_site(g, sub, nsub, L, t);
          cplx<double> a[12], b[12];
          load_site_rw<double, 12>(vj, V, i, a);
          load_site_rw<double, 12>(vl, V, i, b);
          for (int k = 0; k < 12; ++k) b[k] -= cc * a[k];
          store_site<double, 12>(vl, V, i, b);
        }
        __syncthreads();
      }
    double n1 = 0;
    for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
      cplx<double> a[12];
      load_site_rw<double, 12>(vl, V, dfl_site(g, sub, nsub, L, t), a);
      for (int k = 0; k < 12; ++k) n1 += norm2(a[k]);
    }
    n1 = sqrt(block_sum(n1, sh));
    if (!(n1 > 1e-12 * n0)) {
      if (threadIdx.x == 0) atomicExch(rank_loss, 1);
      n1 = 1.0;
    }
    double s = 1.0 / n1;
    for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
      long long i = dfl_site(g, sub, nsub, L, t);
      cplx<double> a[12];
      load_site_rw<double, 12>(vl, V, i, a);
      for (int k = 0; k < 12; ++k) a[k] = s * a[k];
      store_site<double, 12>(vl, V, i, a);
    }
    __syncthreads();
  }
}

// FP64 -> (FP32 ->) BF16, round to nearest even; the FP64 copy takes the rounded values
__global__ void quantize_kernel(size_t V, int Ns, double* b64, uint4* b16) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= V * Ns) return;
  int l = (int)(t / V);
  size_t i = t % V;
  cplx<double> a[12];
  load_site_rw<double, 12>(b64 + (size_t)l * 24 * V, V, i, a);
  for (int u = 0; u < 3; ++u) {
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
    for (int j = 0; j < 4; ++j) {
      cplx<double>& z = a[4 * u + j];
      h[j] = __floats2bfloat162_rn((float)z.re, (float)z.im);
      float2 f = __bfloat1622float2(h[j]);
      z = {(double)f.x, (double)f.y};
    }
    b16[((size_t)l * 3 + u) * V + i] = q;
  }
  store_site<double, 12>(b64 + (size_t)l * 24 * V, V, i, a);
}

// b64 = the BF16 basis b16 in FP64 (inverse of the storage step of quantize_kernel)
__global__ void dequantize_kernel(size_t V, int Ns, const uint4* __restrict__ b16, double* b64) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= V * Ns) return;
  int l = (int)(t / V);
  size_t i = t % V;
  cplx<double> a[12];
  for (int u = 0; u < 3; ++u) {
    cplx<float> c4[4];
    bf16_unpack4(b16[((size_t)l * 3 + u) * V + i], c4);
    for (int j = 0; j < 4; ++j) a[4 * u + j] = {(double)c4[j].re, (double)c4[j].im};
  }
  store_site<double, 12>(b64 + (size_t)l * 24 * V, V, i, a);
}

// ------------------------------------------------------------------ restrict / prolong
// c[L][k] = (phi^L_k, psi)
template <typename T>
__global__ void __launch_bounds__(128) restrict_kernel(Geom g, const int* __restrict__ sub, int nsub, int Ns,
                                                       const double* b64, const uint4* b16,
                                                       const T* __restrict__ psi0, T* __restrict__ c0, int nrhs,
                                                       size_t fstride, size_t cstride) {
  __shared__ T sh[2][NSMAX][4];
  const int L = blockIdx.x;
  const size_t V = g.V;
  const int nsite = nsub * g.svol;
  // the right-hand sides of a batch are handled by the same CTA so the block's basis stays in L2
  for (int rhs = 0; rhs < nrhs; ++rhs) {
  const T* psi = psi0 + (size_t)rhs * fstride;
  T* c = c0 + (size_t)rhs * cstride;
  cplx<T> acc[NSMAX];
#pragma unroll
  for (int k = 0; k < NSMAX; ++k) acc[k] = {T(0), T(0)};
  for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
    long long i = dfl_site(g, sub, nsub, L, t);
    cplx<T> p[12], f[12];
    load_site<T, 12>(psi, V, i, p);
#pragma unroll
    for (int k = 0; k < NSMAX; ++k) {
      if (k < Ns) {
        load_basis<T>(b64, b16, V, k, i, f);
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[k] += cmulc(f[j], p[j]);
      }
    }
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NSMAX; ++k) {
    if (k < Ns) {
      T re = acc[k].re, im = acc[k].im;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) { sh[0][k][w] = re; sh[1][k][w] = im; }
    }
  }
  __syncthreads();
  if (threadIdx.x < Ns) {
    int k = threadIdx.x;
    T re = sh[0][k][0], im = sh[1][k][0];
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j) { re += sh[0][k][j]; im += sh[1][k][j]; }
    c[2 * ((size_t)L * Ns + k)] = re;
    c[2 * ((size_t)L * Ns + k) + 1] = im;
  }
  __syncthreads();
  }
}

// Warp sum of M values per lane by recursive halving: at each butterfly step a lane keeps
// one half of its values, sends the other half to its partner and adds what it receives, so
// M values cost about M shuffles instead of 5 M.  When M becomes odd the remaining steps
// exchange all values.  On return x[0..M_final) holds the warp sums of the values
// base, ..., base + M_final - 1 (base depends on the lane; lanes that differ only in the
// bits of the full-exchange steps hold the same values).  Fixed order: deterministic.
template <typename T, int M, int O>
struct WarpHalve {
  __host__ __device__ static constexpr int final_m() {
    if constexpr (O == 0) return M;
    else if constexpr (M % 2 == 0) return WarpHalve<T, M / 2, O / 2>::final_m();
    else return WarpHalve<T, M, O / 2>::final_m();
  }
  static DW_D void run(T* x, int lane, int& base) {
    if constexpr (O == 0) {
      return;
    } else if constexpr (M % 2 == 0) {
      constexpr int H = M / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const T send = up ? x[i] : x[i + H];
        const T keep = up ? x[i + H] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if (up) base += H;
      WarpHalve<T, H, O / 2>::run(x, lane, base);
    } else {
#pragma unroll
      for (int i = 0; i < M; ++i) x[i] += __shfl_xor_sync(0xffffffffu, x[i], O);
      WarpHalve<T, M, O / 2>::run(x, lane, base);
    }
  }
};

// c[L][k] = (phi^L_k, psi), Ns known at compile time: CTA per deflation block, per-thread
// partial sums in the working precision, CTA sum by warp halving + shared memory.
template <typename T, int NS>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) restrict_ns_kernel(Geom g, const int* __restrict__ sub, int nsub,
                                                             const double* b64, const uint4* b16,
                                                             const T* __restrict__ psi0, T* __restrict__ c0,
                                                             int nrhs, size_t fstride, size_t cstride) {
  using WH = WarpHalve<T, 2 * NS, 16>;
  constexpr int MF = WH::final_m();
  __shared__ T sh[4][2 * NS];
  const int L = blockIdx.x;
  const size_t V = g.V;
  const int nsite = nsub * g.svol;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    const T* psi = psi0 + (size_t)rhs * fstride;
    T* c = c0 + (size_t)rhs * cstride;
    T acc[2 * NS];
#pragma unroll
    for (int k = 0; k < 2 * NS; ++k) acc[k] = T(0);
    for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
      const long long i = dfl_site(g, sub, nsub, L, t);
      cplx<T> p[12];
      load_site<T, 12>(psi, V, i, p);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        cplx<T> f[12];
        load_basis<T>(b64, b16, V, k, i, f);
        T re = 0, im = 0;
#pragma unroll
        for (int j = 0; j < 12; ++j) {
          re += f[j].re * p[j].re + f[j].im * p[j].im;
          im += f[j].re * p[j].im - f[j].im * p[j].re;
        }
        acc[2 * k] += re;
        acc[2 * k + 1] += im;
      }
    }
    int base = 0;
    WH::run(acc, lane, base);
    // lanes holding the same index block hold equal sums; all of them store
#pragma unroll
    for (int m = 0; m < MF; ++m) sh[w][base + m] = acc[m];
    __syncthreads();
    if (threadIdx.x < 2 * NS) {
      T y = sh[0][threadIdx.x];
#pragma unroll
      for (int q = 1; q < 4; ++q) y += sh[q][threadIdx.x];
      c[(size_t)L * 2 * NS + threadIdx.x] = y;
    }
    __syncthreads();
  }
}

// psi = mode 0: Phi c ; 1: psi + Phi c ; 2: psi - Phi c
template <typename T>
__global__ void __launch_bounds__(128) prolong_kernel(Geom g, const int* __restrict__ sap2dfl, int Ns,
                                                      const double* b64, const uint4* b16,
                                                      const T* __restrict__ c0, T* psi0, int mode, int nrhs,
                                                      size_t fstride, size_t cstride) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  const size_t V = g.V;
  const int L = __ldg(sap2dfl + (int)(i >> g.lsvol));
  for (int rhs = 0; rhs < nrhs; ++rhs) {
  const T* c = c0 + (size_t)rhs * cstride;
  T* psi = psi0 + (size_t)rhs * fstride;
  cplx<T> out[12], f[12];
  if (mode == 0) {
#pragma unroll
    for (int j = 0; j < 12; ++j) out[j] = {T(0), T(0)};
  } else {
    load_site_rw<T, 12>(psi, V, i, out);
  }
  const cplx<T>* cc = reinterpret_cast<const cplx<T>*>(c) + (size_t)L * Ns;
  for (int k = 0; k < Ns; ++k) {
    cplx<T> ck = cc[k];
    if (mode == 2) ck = -ck;
    load_basis<T>(b64, b16, V, k, i, f);
#pragma unroll
    for (int j = 0; j < 12; ++j) out[j] += ck * f[j];
  }
  store_site<T, 12>(psi, V, i, out);
  }
}

// ------------------------------------------------------------------ little operator assembly (A.1), FP64
// CTA (L, l, part): part 0: (phi^L_k, D_L phi^L_l) with D_L the deflation-block (Dirichlet) operator;
// part 1+d: (phi^L_k, hop_d phi^{nb(L,d)}_l) over the face of L in direction d.
template <int MU>
DW_D void part_dir(const Geom& g, const SiteRef& s, long long i, const double* __restrict__ links,
                   const double* __restrict__ f, const int* __restrict__ sap2dfl, int myL, int sel,
                   cplx<double>* acc) {
  // sel: -1 -> all hops staying inside the deflation block; d -> only direction d if it leaves the block
  for (int dir = 0; dir < 2; ++dir) {
    int d = 2 * MU + dir;
    if (sel >= 0 && sel != d) continue;
    bool cr;
    long long j = neighbour(g, s, d, &cr);
    int nL = cr ? __ldg(sap2dfl + (int)(j >> g.lsvol)) : myL;
    bool inside = nL == myL;
    if ((sel < 0) != inside) continue;
    double sg = time_wrap(g, s, d) ? -1.0 : 1.0;
    SU3<double> U;
    cplx<double> p[12];
    load_link(links, g.V, MU, dir == 0 ? i : j, U);
    load_site<double, 12>(f, g.V, j, p);
    if (dir == 0) hop_acc<MU, -1, false>(acc, p, U, sg);
    else hop_acc<MU, +1, true>(acc, p, U, sg);
  }
}

__global__ void __launch_bounds__(128) assemble_kernel(Geom g, const int* __restrict__ sub, int nsub,
                                                       const int* __restrict__ sap2dfl, int Ns,
                                                       const double* __restrict__ links,
                                                       const double* __restrict__ clov,
                                                       const double* __restrict__ basis, double* B) {
  __shared__ double sh[2][NSMAX][4];
  const int l = blockIdx.x % Ns;
  const int part = (blockIdx.x / Ns) % 9;
  const int L = blockIdx.x / (9 * Ns);
  const size_t V = g.V;
  const int nsite = nsub * g.svol;
  const double* fl = basis + (size_t)l * 24 * V;
  cplx<double> acc[NSMAX];
  for (int k = 0; k < NSMAX; ++k) acc[k] = {0.0, 0.0};
  for (int t = threadIdx.x; t < nsite; t += blockDim.x) {
    long long i = dfl_site(g, sub, nsub, L, t);
    SiteRef s = decode(g, i);
    cplx<double> w[12], h[12];
    for (int j = 0; j < 12; ++j) h[j] = {0.0, 0.0};
    int sel = part - 1;
    part_dir<0>(g, s, i, links, fl, sap2dfl, L, sel, h);
    part_dir<1>(g, s, i, links, fl, sap2dfl, L, sel, h);
    part_dir<2>(g, s, i, links, fl, sap2dfl, L, sel, h);
    part_dir<3>(g, s, i, links, fl, sap2dfl, L, sel, h);
    bool any = false;
    for (int j = 0; j < 12; ++j) {
      w[j] = -0.5 * h[j];
      any |= (h[j].re != 0.0 || h[j].im != 0.0);
    }
    if (part == 0) {
      cplx<double> p[12], y[12];
      load_site<double, 12>(fl, V, i, p);
      clover_apply(clov, V, i, p, y);
      for (int j = 0; j < 12; ++j) w[j] += y[j];
      any = true;
    }
    if (!any) continue;
    for (int k = 0; k < Ns; ++k) {
      cplx<double> f[12];
      load_site<double, 12>(basis + (size_t)k * 24 * V, V, i, f);
      for (int j = 0; j < 12; ++j) acc[k] += cmulc(f[j], w[j]);
    }
  }
  int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int k = 0; k < Ns; ++k) {
    double re = acc[k].re, im = acc[k].im;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) { sh[0][k][wp] = re; sh[1][k][wp] = im; }
  }
  __syncthreads();
  if (threadIdx.x < Ns) {
    int k = threadIdx.x;
    double re = 0, im = 0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { re += sh[0][k][j]; im += sh[1][k][j]; }
    size_t off = ((((size_t)L * 9 + part) * Ns + l) * Ns + k) * 2;
    B[off] = re;
    B[off + 1] = im;
  }
}

// one CTA (32 threads) per block: Gauss-Jordan inverse of B_LL with partial pivoting in shared
// memory (column-major in and out) and the 1-norm condition number ||B||_1 ||B^{-1}||_1
__global__ void __launch_bounds__(32) block_inverse_kernel(int Ns, const double* __restrict__ B, double* Binv64,
                                                           float* Binv32, double* cond) {
  __shared__ cplx<double> A[NSMAX][NSMAX + 1], X[NSMAX][NSMAX + 1];
  __shared__ int piv_s;
  __shared__ bool sing;
  const int L = blockIdx.x, t = threadIdx.x;
  const double* src = B + (size_t)L * 9 * Ns * Ns * 2;
  double colsum = 0;
  if (t < Ns)
    for (int row = 0; row < Ns; ++row) {
      A[row][t] = {src[2 * (t * Ns + row)], src[2 * (t * Ns + row) + 1]};
      X[row][t] = {row == t ? 1.0 : 0.0, 0.0};
      colsum += sqrt(norm2(A[row][t]));
    }
  double n1 = colsum;
  for (int o = 16; o > 0; o >>= 1) n1 = fmax(n1, __shfl_xor_sync(0xffffffffu, n1, o));
  if (t == 0) sing = false;
  __syncwarp();
  for (int c = 0; c < Ns; ++c) {
    // pivot: largest |A[r][c]|, r >= c
    double v = (t >= c && t < Ns) ? norm2(A[t][c]) : -1.0;
    int r = t;
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      int r2 = __shfl_xor_sync(0xffffffffu, r, o);
      if (v2 > v || (v2 == v && r2 < r)) { v = v2; r = r2; }
    }
    if (t == 0) { piv_s = r; if (!(v > 0.0)) sing = true; }
    __syncwarp();
    if (sing) break;
    int pv = piv_s;
    if (pv != c && t < Ns) {
      cplx<double> tmp = A[c][t]; A[c][t] = A[pv][t]; A[pv][t] = tmp;
      tmp = X[c][t]; X[c][t] = X[pv][t]; X[pv][t] = tmp;
    }
    __syncwarp();
    cplx<double> p = A[c][c];
    double pn = norm2(p);
    cplx<double> pinv = {p.re / pn, -p.im / pn};
    __syncwarp();
    if (t < Ns) { A[c][t] = A[c][t] * pinv; X[c][t] = X[c][t] * pinv; }
    __syncwarp();
    if (t < Ns && t != c) {
      cplx<double> f = A[t][c];
      for (int b2 = 0; b2 < Ns; ++b2) { A[t][b2] -= f * A[c][b2]; X[t][b2] -= f * X[c][b2]; }
    }
    __syncwarp();
  }
  double ni = 0;
  if (t < Ns)
    for (int row = 0; row < Ns; ++row) {
      size_t o = (((size_t)L * Ns + t) * Ns + row) * 2;
      Binv64[o] = X[row][t].re;
      Binv64[o + 1] = X[row][t].im;
      Binv32[o] = (float)X[row][t].re;
      Binv32[o + 1] = (float)X[row][t].im;
      ni += sqrt(norm2(X[row][t]));
    }
  for (int o = 16; o > 0; o >>= 1) ni = fmax(ni, __shfl_xor_sync(0xffffffffu, ni, o));
  if (t == 0) cond[L] = sing ? INFINITY : n1 * ni;
}

// M[L][d] = Binv[L] * B[L][1+d]   (column-major, thread per entry)
__global__ void neighbour_products_kernel(int Nb, int Ns, const double* __restrict__ B,
                                          const double* __restrict__ Binv, double* M64, float* M32) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t total = (size_t)Nb * 8 * Ns * Ns;
  if (t >= total) return;
  int row = (int)(t % Ns);
  int col = (int)((t / Ns) % Ns);
  int d = (int)((t / ((size_t)Ns * Ns)) % 8);
  int L = (int)(t / ((size_t)Ns * Ns * 8));
  const double* bi = Binv + (size_t)L * Ns * Ns * 2;
  const double* bd = B + ((size_t)L * 9 + 1 + d) * Ns * Ns * 2;
  cplx<double> s = {0, 0};
  for (int j = 0; j < Ns; ++j) {
    cplx<double> a = {bi[2 * (j * Ns + row)], bi[2 * (j * Ns + row) + 1]};
    cplx<double> b = {bd[2 * (col * Ns + j)], bd[2 * (col * Ns + j) + 1]};
    s += a * b;
  }
  M64[2 * t] = s.re;
  M64[2 * t + 1] = s.im;
  M32[2 * t] = (float)s.re;
  M32[2 * t + 1] = (float)s.im;
}

// ------------------------------------------------------------------ little vector kernels
// acc(lane) += sum_col m[col*Ns + lane] * sv[col] for lane < Ns.  The source vector is read
// once (one element per lane) and broadcast by warp shuffles; with NS fixed at compile time the
// column loop is unrolled so the coalesced matrix loads are all in flight together.
template <typename T, int NS>
DW_D cplx<T> warp_mv(const cplx<T>* __restrict__ m, const cplx<T>* __restrict__ sv, int Ns, int lane,
                     cplx<T> acc) {
  const int n = NS ? NS : Ns;
  const cplx<T> x = lane < n ? sv[lane] : cplx<T>{T(0), T(0)};
  if (NS) {
#pragma unroll
    for (int col = 0; col < (NS ? NS : 1); ++col) {
      cplx<T> xc = {__shfl_sync(0xffffffffu, x.re, col), __shfl_sync(0xffffffffu, x.im, col)};
      if (lane < NS) acc += m[(size_t)col * NS + lane] * xc;
    }
  } else {
    for (int col = 0; col < n; ++col) {
      cplx<T> xc = {__shfl_sync(0xffffffffu, x.re, col), __shfl_sync(0xffffffffu, x.im, col)};
      if (lane < n) acc += m[(size_t)col * n + lane] * xc;
    }
  }
  return acc;
}

// out[i] = base[i] - sum_d M[blk_i][d] src[lnb[i][d]]   (one CTA of 8 warps per block row,
// warp d computes direction d, lane = row of the Ns x Ns blocks; base may be null).
// M column-major: M[((L*8+d)*Ns + col)*Ns + row].
template <typename T, int NS>
__global__ void __launch_bounds__(256) little_hop_kernel(int n, int Ns, const int* __restrict__ list,
                                                         const int* __restrict__ lnb, const T* __restrict__ M,
                                                         const T* __restrict__ src, const T* base, T* out,
                                                         size_t sys_stride_in = 0, size_t sys_stride_out = 0) {
  // blockIdx.y: system of a batch (vectors sys_stride_* reals apart; base strided like src)
  src += blockIdx.y * sys_stride_in;
  if (base) base += blockIdx.y * sys_stride_out;
  out += blockIdx.y * sys_stride_out;
  __shared__ double hop64[8][2 * 32];
  const int r = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= n) return;
  const int ns = NS ? NS : Ns;
  const int L = __ldg(list + r);
  const int j = __ldg(lnb + r * 8 + w);
  const cplx<T>* Mc = reinterpret_cast<const cplx<T>*>(M);
  const cplx<T>* S = reinterpret_cast<const cplx<T>*>(src);
  const cplx<T> acc = warp_mv<T, NS>(Mc + ((size_t)L * 8 + w) * ns * ns, S + (size_t)j * ns, ns, lane,
                                     cplx<T>{T(0), T(0)});
  hop64[w][2 * lane] = (double)acc.re;
  hop64[w][2 * lane + 1] = (double)acc.im;
  __syncthreads();
  if (w == 0 && lane < ns) {
    double re = 0, im = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { re += hop64[q][2 * lane]; im += hop64[q][2 * lane + 1]; }
    cplx<T>* O = reinterpret_cast<cplx<T>*>(out);
    cplx<T> b = base ? reinterpret_cast<const cplx<T>*>(base)[(size_t)r * ns + lane] : cplx<T>{T(0), T(0)};
    O[(size_t)r * ns + lane] = b - cplx<T>{(T)re, (T)im};
  }
}

// out[i] = Binv[blk_i] * src[i]  (compact parity list vectors)
template <typename T, int NS>
__global__ void little_bdiag_kernel(int n, int Ns, const int* __restrict__ list, const T* __restrict__ Binv,
                                    const T* __restrict__ src, T* out, size_t sys_stride = 0) {
  src += blockIdx.y * sys_stride;       // blockIdx.y: system of a batch
  out += blockIdx.y * sys_stride;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n) return;
  const int ns = NS ? NS : Ns;
  const int L = __ldg(list + wid);
  cplx<T> acc = warp_mv<T, NS>(reinterpret_cast<const cplx<T>*>(Binv) + (size_t)L * ns * ns,
                               reinterpret_cast<const cplx<T>*>(src) + (size_t)wid * ns, ns, lane,
                               cplx<T>{T(0), T(0)});
  if (lane < ns) reinterpret_cast<cplx<T>*>(out)[(size_t)wid * ns + lane] = acc;
}

// run CALL with a compile-time NSV for the common subspace sizes (0 = runtime size)
#define NS_DISPATCH(NSRT, CALL)                                   \
  switch (NSRT) {                                                 \
    case 8: { constexpr int NSV = 8; CALL; } break;               \
    case 12: { constexpr int NSV = 12; CALL; } break;             \
    case 16: { constexpr int NSV = 16; CALL; } break;             \
    case 20: { constexpr int NSV = 20; CALL; } break;             \
    case 24: { constexpr int NSV = 24; CALL; } break;             \
    case 32: { constexpr int NSV = 32; CALL; } break;             \
    default: { constexpr int NSV = 0; CALL; } break;              \
  }

// the same for the largest kernels (FP64 cooperative solver, double-float restriction, multi-RHS
// solver): specialised for Ns = 8 and the paper's Ns = 20 only, the generic kernel otherwise,
// which keeps the library's compile time down
#define NS_DISPATCH_FEW(NSRT, CALL)                               \
  switch (NSRT) {                                                 \
    case 8: { constexpr int NSV = 8; CALL; } break;               \
    case 20: { constexpr int NSV = 20; CALL; } break;             \
    default: { constexpr int NSV = 0; CALL; } break;              \
  }

// gather a parity part of a full little vector ([Nb][Ns]) into compact order / scatter back
template <typename Tin, typename Tout>
__global__ void little_gather_kernel(int n, int Ns, const int* __restrict__ list, const Tin* __restrict__ full,
                                     Tout* part, size_t sys_stride_full = 0, size_t sys_stride_part = 0) {
  full += blockIdx.y * sys_stride_full;   // blockIdx.y: system of a batch
  part += blockIdx.y * sys_stride_part;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * Ns) return;
  int i = t / Ns, k = t % Ns;
  size_t src = ((size_t)list[i] * Ns + k) * 2;
  part[2 * (size_t)t] = (Tout)full[src];
  part[2 * (size_t)t + 1] = (Tout)full[src + 1];
}
template <typename Tin, typename Tout>
__global__ void little_scatter_kernel(int n, int Ns, const int* __restrict__ list, const Tin* __restrict__ part,
                                      Tout* full, size_t sys_stride_part = 0, size_t sys_stride_full = 0) {
  part += blockIdx.y * sys_stride_part;   // blockIdx.y: system of a batch
  full += blockIdx.y * sys_stride_full;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * Ns) return;
  int i = t / Ns, k = t % Ns;
  size_t dst = ((size_t)list[i] * Ns + k) * 2;
  full[dst] = (Tout)part[2 * (size_t)t];
  full[dst + 1] = (Tout)part[2 * (size_t)t + 1];
}

// full little operator w = A v (FP64), one warp per block
__global__ void little_full_kernel(int Nb, int Ns, const int* __restrict__ bnb, const double* __restrict__ B,
                                   const double* __restrict__ v, double* w) {
  int L = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (L >= Nb) return;
  const cplx<double>* Bc = reinterpret_cast<const cplx<double>*>(B);
  const cplx<double>* vc = reinterpret_cast<const cplx<double>*>(v);
  cplx<double> acc = {0, 0};
  for (int part = 0; part < 9; ++part) {
    int src = part == 0 ? L : bnb[L * 8 + part - 1];
    const cplx<double>* m = Bc + ((size_t)L * 9 + part) * Ns * Ns;
    for (int col = 0; col < Ns; ++col) {
      cplx<double> x = vc[(size_t)src * Ns + col];
      if (lane < Ns) acc += m[(size_t)col * Ns + lane] * x;
    }
  }
  if (lane < Ns) reinterpret_cast<cplx<double>*>(w)[(size_t)L * Ns + lane] = acc;
}

inline unsigned warps_grid(int n, int threads = 128) { return (unsigned)((n * 32 + threads - 1) / threads); }

}  // namespace

// ------------------------------------------------------------------ cooperative little GCR (A.2-A.4)
// The whole even-odd, globally deflated little GCR in one persistent kernel:
// grid-wide barriers replace the host round trips of the host-driven loop.
// Ownership: CTA c owns the contiguous range of block rows [c R, (c+1) R) of
// each parity, and with its even rows the entries of every even-site little
// vector on them, so the even hop and all elementwise work and inner products
// that follow it stay inside the CTA.  Reductions: per-CTA sums in shared
// memory, added in FP64 into one of three rotating global accumulators, a grid
// barrier, then every CTA reads the totals (the FP64 sum of FP32 partials is
// exact enough that the FP32 results do not depend on the order of the adds).
// Inner products with many vectors are CTA-slice GEMVs: warp w owns the vectors
// j = w, w + 8, ...  One GCR step takes three grid barriers: after the odd hop,
// and two reductions (the A.3 projection and the Gram-Schmidt coefficients share
// one, with the coefficients of the projected vector obtained from those of the
// raw vector and a table of (chi_j, B^ g_l); the second gives c_k, a_k and the
// table row).  The residual rho_{k+1} = rho_k - (a_k / c_k) chi'_k is not
// published before the next step: rho is double-buffered and chi'_k kept
// unnormalised, so the next odd hop forms rho_{k+1} on the fly from two vectors
// every CTA can read after the second reduction; |rho_{k+1}|^2 is folded into
// the next step's first reduction (the stopping test of a step uses
// |rho_k|^2 - |a_k|^2 and the cycle end recomputes the true residual).
constexpr int COOP_THREADS = 256;
constexpr int COOP_WARPS = COOP_THREADS / 32;
constexpr int COOP_NV = 128;         // values per grid reduction
constexpr int COOP_NKV = 24;         // Krylov vectors per cycle
constexpr int COOP_CH = 16;          // block rows per hop chunk
#ifndef COOP_HOP_DEPTH
#define COOP_HOP_DEPTH 2             // rows in flight per warp in the FP32 hops
#endif

template <typename T>
struct CoopArgs {
  int Ne, No, Ns, nkv, maxit, a3;
  const int *list_e, *list_o, *lnb_e, *lnb_o;
  const T *M, *g, *Bg, *Ainv, *b;
  T* v;
  T* work;            // (2 nkv + 5) vectors of Ne*Ns complex
  double* acc;        // [3][COOP_NV] reduction accumulators, zero at launch
  double* out;        // [0] iterations, [1] relative residual
  int* err;           // set when a bounded wait of the shared-memory ring gave up
  int vec_rows;       // > 0: this CTA's slices of g, B^ g and chi'_j (vec_rows block rows each) are kept
                      // in dynamic shared memory after the hop partial sums (register-pipelined hops)
  double tol;
};

// Shared state of one CTA.  All arithmetic of the solver runs in the working precision T:
// FP32 throughput is many times that of FP64 on this part, and the FP32 solve is a
// preconditioner-level solve whose residual is recomputed in FP64 by the caller.
template <typename T>
struct CoopShared {
  T ws[COOP_WARPS][4];
  T cta[COOP_NV];            // this CTA's share of the values being reduced
  T res[COOP_NV];            // grid-wide sums
  T a[2 * COOP_NKV], c[COOP_NKV], beta[2 * COOP_NKV];
  T bb[COOP_NKV][2 * COOP_NKV];
  T tg[COOP_NKV][2 * 32];    // (chi_j, B^ g_l) of the current cycle's chi_j (normalised chi_j)
  T z[2 * 32];
  T ainv[2 * 32 * 32];       // A~^{-1}, row-major
  T ac[2];                   // a_{k-1} / c_{k-1}: rho_k = rho_{k-1} - ac chi'_{k-1}
  T bbn[2 * COOP_NKV];       // b_jk / c_j of the current step (coefficients on the unnormalised chi'_j)
  T rr;                      // this CTA's share of |rho_k|^2 (folded into the next reduction)
  int phase;
};

// row stride of the partial-sum table of the multi-RHS solver: a multiple of 4 (16-byte loads)
DW_HD int coop_gpad(int grid) { return (grid + 3) & ~3; }

// dynamic shared memory of the cooperative kernel: hop partial sums
template <typename T>
inline size_t coop_dyn_smem(int) {
  return (size_t)COOP_CH * 8 * 64 * sizeof(T);
}

struct CoopSlice {
  size_t s0, s1;
};

// entries of the even-site little vectors on this CTA's even block rows
DW_D CoopSlice coop_rows_slice(int nrow, int ns) {
  const int R = (nrow + gridDim.x - 1) / gridDim.x;
  const int rb = min(nrow, (int)blockIdx.x * R), re = min(nrow, rb + R);
  return {(size_t)rb * ns, (size_t)re * ns};
}

template <typename T>
DW_D T warp_allsum(T y) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
  return y;
}

// Sum the nv values sh.cta[0..nv) over all CTAs; result in sh.res (all CTAs).  Each CTA adds
// its values in FP64 into accumulator set (phase mod 3); after the barrier every CTA reads the
// totals past L1.  CTA 0 clears the set used two reductions ahead: that set was last read
// before this barrier and is next added to after the following one.
template <typename T>
DW_D void coop_reduce(cg::grid_group& grid, CoopShared<T>& sh, int nv, double* acc_base) {
  __syncthreads();
  double* acc = acc_base + (size_t)(sh.phase % 3) * COOP_NV;
  if (threadIdx.x < nv) atomicAdd(acc + threadIdx.x, (double)sh.cta[threadIdx.x]);
  __syncthreads();
  grid.sync();
  if (threadIdx.x < nv) sh.res[threadIdx.x] = (T)__ldcg(acc + threadIdx.x);
  if (blockIdx.x == 0 && threadIdx.x < COOP_NV) acc_base[(size_t)((sh.phase + 2) % 3) * COOP_NV + threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) sh.phase += 1;
  __syncthreads();
}

// per-thread values x[0..NV) -> their CTA sums in sh.cta[0..NV)
template <typename T, int NV>
DW_D void cta_sum(CoopShared<T>& sh, T (&x)[NV]) {
  static_assert(NV <= 4, "few values only");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const T y = warp_allsum(x[j]);
    if (lane == 0) sh.ws[w][j] = y;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T y = 0;
#pragma unroll
    for (int q = 0; q < COOP_WARPS; ++q) y += sh.ws[q][threadIdx.x];
    sh.cta[threadIdx.x] = y;
  }
}

// sh.cta[off + 2j], sh.cta[off + 2j + 1] = this CTA's share of (X_j, y) for j < nvec;
// X_j = X + j xstride.  Starts with a CTA barrier (y may have been written by other
// threads of the CTA).
template <typename T>
DW_D void cta_dots(CoopShared<T>& sh, const cplx<T>* X, size_t xstride, int nvec, const cplx<T>* y,
                   const CoopSlice& sl, int off) {
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // four vectors per warp and pass (j0 + 8u), so that their loads are in flight together;
  // the eight sums of a warp are reduced by recursive halving
  for (int j0 = w; j0 < nvec; j0 += 4 * COOP_WARPS) {
    const cplx<T>* xs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jj = j0 + u * COOP_WARPS;
      xs[u] = X + (size_t)(jj < nvec ? jj : j0) * xstride;
    }
    T acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = 0;
#pragma unroll 4
    for (size_t i = sl.s0 + lane; i < sl.s1; i += 32) {
      const cplx<T> q = y[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const cplx<T> p = xs[u][i];
        acc[2 * u] += p.re * q.re + p.im * q.im;
        acc[2 * u + 1] += p.re * q.im - p.im * q.re;
      }
    }
    int base = 0;
    WarpHalve<T, 8, 16>::run(acc, lane, base);     // lane holds the sum of value 'base'
    const int u = base >> 1, jj = j0 + u * COOP_WARPS;
    if ((lane & 3) == 0 && jj < nvec) sh.cta[off + 2 * jj + (base & 1)] = acc[0];
  }
}

// Ns x Ns block times vector, loads issued up front: lane = output row, x broadcast by shuffles.
// The vector is src - cs * corr when corr is given (the residual formed on the fly).
template <typename T, int NS>
struct RowLoad {
  cplx<T> m[NS];
  cplx<T> x;
  DW_D void load(const cplx<T>* __restrict__ Mb, const cplx<T>* __restrict__ sv, const cplx<T>* __restrict__ cv,
                 cplx<T> cs, int lane) {
#pragma unroll
    for (int c = 0; c < NS; ++c) m[c] = lane < NS ? Mb[c * NS + lane] : cplx<T>{T(0), T(0)};
    x = lane < NS ? sv[lane] : cplx<T>{T(0), T(0)};
    if (cv && lane < NS) x -= cs * cv[lane];
  }
  DW_D cplx<T> mv() const {
    cplx<T> acc = {T(0), T(0)};
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      const cplx<T> xc = {__shfl_sync(0xffffffffu, x.re, c), __shfl_sync(0xffffffffu, x.im, c)};
      acc += m[c] * xc;
    }
    return acc;
  }
};

// out[r] = base[r] + out_sign * sum_d M[list[r]][d] (src - cs corr)[lnb[r][d]] for this CTA's block
// rows (corr may be null).  Rows in chunks of COOP_CH; warp d computes direction d of every row of
// the chunk (FP32: the next row's block is loaded while the current one is multiplied), the 8
// partial sums meet in shared memory (hp, COOP_CH x 8 x 32 complex).
template <typename T, int NS>
DW_D void coop_hop(int nrow, int Ns, const int* list, const int* lnb, const T* M, const cplx<T>* src,
                   const cplx<T>* corr, cplx<T> cs, const cplx<T>* base, cplx<T>* out, T out_sign, cplx<T>* hp) {
  const int ns = NS ? NS : Ns;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const cplx<T>* Mc = reinterpret_cast<const cplx<T>*>(M);
  const int R = (nrow + gridDim.x - 1) / gridDim.x;
  const int rb = min(nrow, (int)blockIdx.x * R), re = min(nrow, rb + R);
  constexpr bool PIPE = sizeof(T) == 4 && NS > 0 && NS <= 24;
  for (int r0 = rb; r0 < re; r0 += COOP_CH) {
    const int nr = min(COOP_CH, re - r0);
    int myL = 0, myj = 0;
    if (lane < nr) { myL = list[r0 + lane]; myj = lnb[(r0 + lane) * 8 + w]; }
    if constexpr (PIPE) {
      // rolling register pipeline: the blocks of the next COOP_HOP_DEPTH - 1 rows are in flight
      // while the current row is multiplied
      constexpr int NB = COOP_HOP_DEPTH;
      RowLoad<T, (PIPE ? NS : 1)> buf[NB];
      auto load_row = [&](RowLoad<T, (PIPE ? NS : 1)>& b, int q) {
        const size_t j = (size_t)__shfl_sync(0xffffffffu, myj, q) * NS;
        b.load(Mc + ((size_t)__shfl_sync(0xffffffffu, myL, q) * 8 + w) * NS * NS, src + j, corr ? corr + j : nullptr,
               cs, lane);
      };
#pragma unroll
      for (int u = 0; u < NB - 1; ++u)
        if (u < nr) load_row(buf[u], u);
      for (int q0 = 0; q0 < nr; q0 += NB) {
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int q = q0 + u;
          if (q < nr) {
            if (q + NB - 1 < nr) load_row(buf[(u + NB - 1) % NB], q + NB - 1);
            hp[(q * 8 + w) * 32 + lane] = buf[u].mv();
          }
        }
      }
    } else {
      for (int q = 0; q < nr; ++q) {
        const int L = __shfl_sync(0xffffffffu, myL, q), j = __shfl_sync(0xffffffffu, myj, q);
        const cplx<T>* m = Mc + ((size_t)L * 8 + w) * ns * ns;
        cplx<T> x = lane < ns ? src[(size_t)j * ns + lane] : cplx<T>{T(0), T(0)};
        if (corr && lane < ns) x -= cs * corr[(size_t)j * ns + lane];
        cplx<T> acc = {T(0), T(0)};
        for (int col = 0; col < ns; ++col) {
          const cplx<T> xc = {__shfl_sync(0xffffffffu, x.re, col), __shfl_sync(0xffffffffu, x.im, col)};
          if (lane < ns) acc += m[(size_t)col * ns + lane] * xc;
        }
        hp[(q * 8 + w) * 32 + lane] = acc;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * ns; t += COOP_THREADS) {
      const int q = t / ns, k = t - q * ns;
      cplx<T> sum = hp[(q * 8) * 32 + k];
#pragma unroll
      for (int d = 1; d < 8; ++d) sum += hp[(q * 8 + d) * 32 + k];
      const size_t o = (size_t)(r0 + q) * ns + k;
      const cplx<T> bse = base ? base[o] : cplx<T>{T(0), T(0)};
      out[o] = bse + out_sign * sum;
    }
    __syncthreads();
  }
}

// The hops with the operator staged in shared memory: the 8 blocks of a block row (8 Ns^2 complex,
// contiguous) arrive by one bulk copy into a ring of RING_SLOTS slots (full barrier: bytes landed;
// empty barrier: the 8 warps are done with the slot).  Thread 0 keeps RING_SLOTS rows in flight and,
// at the end of a hop, issues the first rows of the next hop (odd and even hops alternate), so the
// copies overlap the grid barrier and the reductions between hops.  Counters are kept identically
// by every thread; only thread 0 issues copies.
constexpr int RING_SLOTS = 6;
template <int NS>
struct HopRing {
  uint64_t* full;
  uint64_t* empty;
  unsigned char* slots;
  uint32_t prod, cons;     // rows issued / consumed since the kernel started
  int next_issued;         // rows of the coming hop already issued
  int next_parity;         // 1: odd rows come next, 0: even rows
  int* err;
  __host__ __device__ static constexpr uint32_t bytes() { return (uint32_t)(8 * NS * NS * 2 * sizeof(float)); }
  __host__ __device__ static constexpr uint32_t stride() { return (bytes() + 127u) & ~127u; }
};

DW_D void coop_row_range(int nrow, int* rb, int* re) {
  const int R = (nrow + gridDim.x - 1) / gridDim.x;
  *rb = min(nrow, (int)blockIdx.x * R);
  *re = min(nrow, *rb + R);
}

// thread 0: copy block row L into the next slot (after the slot's previous row has been consumed)
template <int NS>
DW_D void ring_issue(HopRing<NS>& rg, const float* M, int L) {
  const uint32_t p = rg.prod, sl = p % RING_SLOTS;
  if (threadIdx.x == 0) {
    if (p >= RING_SLOTS) mbar_wait(&rg.empty[sl], ((p / RING_SLOTS) - 1) & 1, rg.err);
    mbar_expect_tx(&rg.full[sl], HopRing<NS>::bytes());
    bulk_load(rg.slots + (size_t)sl * HopRing<NS>::stride(), M + (size_t)L * 8 * NS * NS * 2, HopRing<NS>::bytes(),
              &rg.full[sl]);
  }
  ++rg.prod;
}

// issue the first rows of the hop over `list` (this CTA's rows) that are not yet in flight
template <int NS>
DW_D void ring_prefetch(HopRing<NS>& rg, const float* M, int nrow, const int* list) {
  int rb, re;
  coop_row_range(nrow, &rb, &re);
  const int want = min(RING_SLOTS, re - rb);
  for (int j = rg.next_issued; j < want; ++j) ring_issue<NS>(rg, M, list[rb + j]);
  rg.next_issued = max(rg.next_issued, want);
}

// as coop_hop (FP32, Ns = NS), the blocks read from the ring; afterwards the first rows of the
// hop over (nrow_next, list_next) are issued
template <int NS>
DW_D void coop_hop_ring(HopRing<NS>& rg, int nrow, const int* list, const int* lnb, const float* M,
                        const cplx<float>* src, const cplx<float>* corr, cplx<float> cs, const cplx<float>* base,
                        cplx<float>* out, float out_sign, cplx<float>* hp, int nrow_next, const int* list_next) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int rb, re;
  coop_row_range(nrow, &rb, &re);
  ring_prefetch<NS>(rg, M, nrow, list);            // normally done at the end of the previous hop
  for (int r0 = rb; r0 < re; r0 += COOP_CH) {
    const int nr = min(COOP_CH, re - r0);
    // the source entries of every row of the chunk (direction w) into the warp's slots of hp: all
    // the gathers are in flight together instead of one L2 round trip per row
    if (lane < NS)
      for (int q = 0; q < nr; ++q) {
        const int j = __ldg(lnb + (size_t)(r0 + q) * 8 + w);
        cplx<float> x = src[(size_t)j * NS + lane];
        if (corr) x -= cs * corr[(size_t)j * NS + lane];
        hp[(q * 8 + w) * 32 + lane] = x;
      }
    __syncwarp();
    for (int q = 0; q < nr; ++q) {
      const uint32_t c = rg.cons, sl = c % RING_SLOTS;
      if (!mbar_wait(&rg.full[sl], (c / RING_SLOTS) & 1, rg.err)) break;
      const cplx<float>* Mb = reinterpret_cast<const cplx<float>*>(rg.slots + (size_t)sl * HopRing<NS>::stride()) +
                              (size_t)w * NS * NS;
      const cplx<float>* xq = hp + (q * 8 + w) * 32;           // broadcast reads
      cplx<float> a0 = {0.f, 0.f}, a1 = {0.f, 0.f};            // two chains of FMAs
      if (lane < NS) {
#pragma unroll
        for (int col = 0; col < NS; col += 2) {
          a0 += Mb[col * NS + lane] * xq[col];
          if (col + 1 < NS) a1 += Mb[(col + 1) * NS + lane] * xq[col + 1];
        }
      }
      __syncwarp();
      hp[(q * 8 + w) * 32 + lane] = a0 + a1;
      __syncwarp();
      if (lane == 0) mbar_arrive(&rg.empty[sl]);
      ++rg.cons;
      // keep RING_SLOTS rows in flight: refill with the row RING_SLOTS ahead
      const int ahead = (r0 + q - rb) + RING_SLOTS;
      if (ahead < re - rb) ring_issue<NS>(rg, M, __ldg(list + rb + ahead));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * NS; t += COOP_THREADS) {
      const int q = t / NS, k = t - q * NS;
      cplx<float> sum = hp[(q * 8) * 32 + k];
#pragma unroll
      for (int d = 1; d < 8; ++d) sum += hp[(q * 8 + d) * 32 + k];
      const size_t o = (size_t)(r0 + q) * NS + k;
      const cplx<float> bse = base ? base[o] : cplx<float>{0.f, 0.f};
      out[o] = bse + out_sign * sum;
    }
    __syncthreads();
  }
  rg.next_issued = 0;
  ring_prefetch<NS>(rg, M, nrow_next, list_next);
}

// y = B^ x = x - M_eo (M_oe x); ends with a grid barrier.  The CTA barriers on both sides of
// the grid barriers are redundant for correctness but halve the solver's run time on GB300
// (measured: 3.8 ms -> 1.9 ms for 42 iterations at Nb = 2592, Ns = 20).
// one hop through the register pipeline or the shared-memory ring (FP32, Ns = NS only)
template <typename T, int NS, bool RING>
DW_D void hop_any(HopRing<(NS > 0 ? NS : 1)>& rg, const CoopArgs<T>& a, bool odd, const cplx<T>* src,
                  const cplx<T>* corr, cplx<T> cs, const cplx<T>* base, cplx<T>* out, T sign, cplx<T>* hp) {
  const int n = odd ? a.No : a.Ne, nn = odd ? a.Ne : a.No;
  const int* list = odd ? a.list_o : a.list_e;
  const int* lnb = odd ? a.lnb_o : a.lnb_e;
  if constexpr (RING && sizeof(T) == 4 && NS > 0) {
    coop_hop_ring<NS>(rg, n, list, lnb, reinterpret_cast<const float*>(a.M), src, corr, cs, base, out, sign, hp, nn,
                      odd ? a.list_e : a.list_o);
  } else {
    coop_hop<T, NS>(n, a.Ns, list, lnb, a.M, src, corr, cs, base, out, sign, hp);
  }
}

template <typename T, int NS, bool RING>
DW_D void coop_bhat(cg::grid_group& grid, HopRing<(NS > 0 ? NS : 1)>& rg, const CoopArgs<T>& a, const cplx<T>* x,
                    cplx<T>* tmpo, cplx<T>* y, cplx<T>* hp) {
  const cplx<T> zero = {T(0), T(0)};
  hop_any<T, NS, RING>(rg, a, true, x, nullptr, zero, nullptr, tmpo, T(1), hp);     // tmpo = M_oe x
  __syncthreads();
  grid.sync();
  __syncthreads();
  hop_any<T, NS, RING>(rg, a, false, tmpo, nullptr, zero, x, y, T(-1), hp);         // y = x - M_eo tmpo
  __syncthreads();
  grid.sync();
  __syncthreads();
}

// z = A~^{-1} u with u = sh.res[0..2 Ns), into sh.z (threads < Ns; no barrier)
template <typename T>
DW_D void coop_z(CoopShared<T>& sh, int Ns) {
  if (threadIdx.x < Ns) {
    T zr = 0, zi = 0;
    for (int q = 0; q < Ns; ++q) {
      const T mr = sh.ainv[2 * (threadIdx.x * Ns + q)], mi = sh.ainv[2 * (threadIdx.x * Ns + q) + 1];
      const T yr = sh.res[2 * q], yi = sh.res[2 * q + 1];
      zr += mr * yr - mi * yi;
      zi += mr * yi + mi * yr;
    }
    sh.z[2 * threadIdx.x] = zr;
    sh.z[2 * threadIdx.x + 1] = zi;
  }
}

// u -= Bg A~^{-1} g^+ u  (P~_L, in place); with add_to set, only z = A~^{-1} g^+ u is formed and
// add_to += g z is applied instead.  Elementwise parts on the CTA's rows, no trailing barrier.
template <typename T, int NS>
DW_D void coop_PL(cg::grid_group& grid, CoopShared<T>& sh, const CoopArgs<T>& a, cplx<T>* u, const cplx<T>* gsrc,
                  const cplx<T>* bgsrc, cplx<T>* add_to, const CoopSlice& sl) {
  constexpr int NSM = NS ? NS : 32;
  const size_t n = (size_t)a.Ne * a.Ns;
  const int Ns = NS ? NS : a.Ns;
  cta_dots<T>(sh, gsrc, n, Ns, u, sl, 0);
  coop_reduce(grid, sh, 2 * Ns, a.acc);
  coop_z(sh, Ns);
  __syncthreads();
  cplx<T>* tgt = add_to ? add_to : u;
  const cplx<T>* vecs = add_to ? gsrc : bgsrc;
  const T sg = add_to ? T(1) : T(-1);
  for (size_t i = sl.s0 + threadIdx.x; i < sl.s1; i += COOP_THREADS) {
    cplx<T> x = tgt[i];
#pragma unroll
    for (int l = 0; l < NSM; ++l) {
      if (l < Ns) {
        const cplx<T> zl = {sh.z[2 * l], sh.z[2 * l + 1]};
        x += sg * (zl * vecs[(size_t)l * n + i]);
      }
    }
    tgt[i] = x;
  }
}

// shared memory of the vector slices (g, B^ g: Ns vectors each; chi'_j: nkv vectors) of a CTA that
// owns `rows` block rows; the register-pipelined kernels are given up to coop_vec_smem_max() bytes
template <typename T>
inline size_t coop_vec_smem(int rows, int Ns, int nkv) {
  return (size_t)(2 * Ns + nkv) * rows * Ns * 2 * sizeof(T);
}
template <typename T>
inline size_t coop_vec_smem_max() { return (sizeof(T) == 4 ? 200 : 180) * 1024; }   // + static CoopShared <= 227 KB

// dynamic shared memory of the ring variant: hop partial sums, the slots, their barriers
template <int NS>
inline size_t coop_ring_smem() {
  return (size_t)COOP_CH * 8 * 64 * sizeof(float) + (size_t)RING_SLOTS * HopRing<NS>::stride() +
         2 * RING_SLOTS * sizeof(uint64_t);
}

template <typename T, int NS, bool RING = false>
__global__ void __launch_bounds__(COOP_THREADS, 1) little_gcr_coop_kernel(CoopArgs<T> a) {
  constexpr int NSM = NS ? NS : 32;
  constexpr int NSR = NS > 0 ? NS : 1;
  cg::grid_group grid = cg::this_grid();
  __shared__ CoopShared<T> sh;
  extern __shared__ __align__(128) unsigned char coop_dyn[];
  cplx<T>* hp = reinterpret_cast<cplx<T>*>(coop_dyn);                // [COOP_CH][8][32]
  HopRing<NSR> rg{};
  if constexpr (RING) {
    unsigned char* base = coop_dyn + (size_t)COOP_CH * 8 * 64 * sizeof(float);
    rg.slots = base;
    rg.full = reinterpret_cast<uint64_t*>(base + (size_t)RING_SLOTS * HopRing<NSR>::stride());
    rg.empty = rg.full + RING_SLOTS;
    rg.err = a.err;
    if (threadIdx.x == 0) {
      for (int q = 0; q < RING_SLOTS; ++q) {
        mbar_init(&rg.full[q], 1);
        mbar_init(&rg.empty[q], COOP_WARPS);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  const int ns = NS ? NS : a.Ns;
  const size_t n = (size_t)a.Ne * ns;
  const CoopSlice sl = coop_rows_slice(a.Ne, ns);
  const int nkv = a.nkv;
  const int na = a.a3 ? 2 * ns : 0;          // reduced values of the A.3 projection
  const cplx<T> zero = {T(0), T(0)};
  if (threadIdx.x == 0) sh.phase = 0;
  if (a.a3) {
    const cplx<T>* Ai = reinterpret_cast<const cplx<T>*>(a.Ainv);
    for (int t = threadIdx.x; t < ns * ns; t += COOP_THREADS) {
      sh.ainv[2 * t] = Ai[t].re;
      sh.ainv[2 * t + 1] = Ai[t].im;
    }
  }
  __syncthreads();
  cplx<T>* W = reinterpret_cast<cplx<T>*>(a.work);
  cplx<T>* rhob[2] = {W + (size_t)2 * nkv * n, W + (size_t)(2 * nkv + 1) * n};
  // shared-memory copies of this CTA's slices (index i - s0): g, B^ g (constant) and chi'_j
  const bool vs = !RING && a.vec_rows > 0;
  const size_t vstr = (size_t)a.vec_rows * ns;
  cplx<T>* gS = reinterpret_cast<cplx<T>*>(coop_dyn + (size_t)COOP_CH * 8 * 64 * sizeof(T));
  cplx<T>* bgS = gS + (size_t)ns * vstr;
  cplx<T>* chiS = bgS + (size_t)ns * vstr;
  if (vs && a.a3) {
    for (size_t e = threadIdx.x; e < (size_t)ns * (sl.s1 - sl.s0); e += COOP_THREADS) {
      const size_t l = e / (sl.s1 - sl.s0), i = sl.s0 + e % (sl.s1 - sl.s0);
      gS[l * vstr + (i - sl.s0)] = reinterpret_cast<const cplx<T>*>(a.g)[l * n + i];
      bgS[l * vstr + (i - sl.s0)] = reinterpret_cast<const cplx<T>*>(a.Bg)[l * n + i];
    }
    __syncthreads();
  }
  // the vectors as seen by the inner products and updates of a step (shifted so that entry i of
  // vector j sits at [j * stride + i] for this CTA's i)
  const cplx<T>* gV = vs ? gS - sl.s0 : reinterpret_cast<const cplx<T>*>(a.g);
  const cplx<T>* bgV = vs ? bgS - sl.s0 : reinterpret_cast<const cplx<T>*>(a.Bg);
  const cplx<T>* chiV = vs ? chiS - sl.s0 : W;
  const size_t vn = vs ? vstr : n;
  cplx<T>* tmpo = W + (size_t)(2 * nkv + 2) * n;
  cplx<T>* t = W + (size_t)(2 * nkv + 3) * n;
  cplx<T>* rhsd = W + (size_t)(2 * nkv + 4) * n;
  const cplx<T>* b = reinterpret_cast<const cplx<T>*>(a.b);
  const cplx<T>* g = reinterpret_cast<const cplx<T>*>(a.g);
  const cplx<T>* Bg = reinterpret_cast<const cplx<T>*>(a.Bg);
  cplx<T>* v = reinterpret_cast<cplx<T>*>(a.v);
  auto chi = [&](int k) { return W + (size_t)k * n; };      // chi'_k, unnormalised (norm c_k)
  auto xi = [&](int k) { return W + (size_t)(nkv + k) * n; };
  auto slice = [&](auto&& f) {
    for (size_t i = sl.s0 + threadIdx.x; i < sl.s1; i += COOP_THREADS) f(i);
  };

  // rhsd = P~_L b, rho = rhsd, v = 0
  int cur = 0;                               // rhob[cur] holds rho_k on this CTA's rows
  slice([&](size_t i) { rhsd[i] = b[i]; });
  if (a.a3) coop_PL<T, NS>(grid, sh, a, rhsd, g, Bg, nullptr, sl);
  T s1[1] = {0};
  slice([&](size_t i) {
    const cplx<T> x = rhsd[i];
    rhob[0][i] = x;
    v[i] = zero;
    s1[0] += x.re * x.re + x.im * x.im;
  });
  cta_sum<T, 1>(sh, s1);
  if (threadIdx.x == 0) sh.rr = sh.cta[0];
  coop_reduce(grid, sh, 1, a.acc);
  const T bn = sqrt(sh.res[0]);
  T rn = bn;
  int total = 0;
  while (bn > 0 && (double)rn > a.tol * (double)bn && total < a.maxit) {
    int k = 0;
    T rn2 = rn * rn;                         // |rho_k|^2 (exact at the start of a cycle)
    for (; k < nkv && total < a.maxit; ++k) {
      cplx<T>* ck = chi(k);
      cplx<T>* xk = xi(k);
      cplx<T>* rk = rhob[cur];
      // xi_k = rho_k;  chi_k = B^ rho_k.  The odd hop reads rho_k of other CTAs as
      // rho_{k-1} - ac chi'_{k-1} (both final since the last reduction); the even hop writes
      // this CTA's own rows, so no grid barrier follows it
      slice([&](size_t i) { xk[i] = rk[i]; });
      const cplx<T> acs = k > 0 ? cplx<T>{sh.ac[0], sh.ac[1]} : zero;
      hop_any<T, NS, RING>(rg, a, true, k > 0 ? rhob[cur ^ 1] : rk, k > 0 ? chi(k - 1) : nullptr, acs, nullptr, tmpo,
                           T(1), hp);
      __syncthreads();
      grid.sync();
      __syncthreads();
      hop_any<T, NS, RING>(rg, a, false, tmpo, nullptr, zero, rk, ck, T(-1), hp);
      // one reduction: u = g^+ chi_k (A.3), the raw coefficients (chi'_j, chi_k), j < k, and |rho_k|^2
      if (a.a3) cta_dots<T>(sh, gV, vn, ns, ck, sl, 0);
      if (k > 0) cta_dots<T>(sh, chiV, vn, k, ck, sl, na);
      __syncthreads();
      if (threadIdx.x == 0) sh.cta[na + 2 * k] = sh.rr;
      coop_reduce(grid, sh, na + 2 * k + 1, a.acc);
      rn2 = sh.res[na + 2 * k];
      rn = sqrt(rn2);
      if ((double)rn <= a.tol * (double)bn) break;    // rho_k already converged: chi_k unused
      if (a.a3) coop_z(sh, ns);
      __syncthreads();
      // coefficients of the projected vector P~_L chi_k on the normalised chi_j:
      // (chi'_j, chi_k) / c_j - sum_l z_l (chi_j, B^ g_l)
      if (threadIdx.x < k) {
        const int j = threadIdx.x;
        const T ic = T(1) / sh.c[j];
        T br = sh.res[na + 2 * j] * ic, bi = sh.res[na + 2 * j + 1] * ic;
        if (a.a3) {
          for (int l = 0; l < ns; ++l) {
            const T zr = sh.z[2 * l], zi = sh.z[2 * l + 1], tr = sh.tg[j][2 * l], ti = sh.tg[j][2 * l + 1];
            br -= zr * tr - zi * ti;
            bi -= zr * ti + zi * tr;
          }
        }
        sh.bb[j][2 * k] = br;
        sh.bb[j][2 * k + 1] = bi;
        sh.bbn[2 * j] = br * ic;
        sh.bbn[2 * j + 1] = bi * ic;
      }
      __syncthreads();
      // chi'_k = P~_L chi_k - sum_j b_jk chi'_j / c_j ; then (chi'_k, rho_k), |chi'_k|^2, (B^ g_l, chi'_k)
      T s3[3] = {0, 0, 0};
      slice([&](size_t i) {
        cplx<T> y = ck[i], y2 = {T(0), T(0)};         // two chains of FMAs
        if (a.a3) {
#pragma unroll
          for (int l = 0; l < NSM; ++l)
            if (l < ns) {
              const cplx<T> t = cplx<T>{sh.z[2 * l], sh.z[2 * l + 1]} * bgV[(size_t)l * vn + i];
              if (l & 1) y2 -= t; else y -= t;
            }
        }
#pragma unroll
        for (int j = 0; j < COOP_NKV; ++j)
          if (j < k) {
            const cplx<T> t = cplx<T>{sh.bbn[2 * j], sh.bbn[2 * j + 1]} * chiV[(size_t)j * vn + i];
            if (j & 1) y2 -= t; else y -= t;
          }
        y += y2;
        ck[i] = y;
        if (vs) chiS[(size_t)k * vstr + (i - sl.s0)] = y;
        const cplx<T> r = rk[i];
        s3[0] += y.re * r.re + y.im * r.im;
        s3[1] += y.re * r.im - y.im * r.re;
        s3[2] += y.re * y.re + y.im * y.im;
      });
      cta_sum<T, 3>(sh, s3);
      if (a.a3) cta_dots<T>(sh, bgV, vn, ns, ck, sl, 3);
      coop_reduce(grid, sh, 3 + na, a.acc);
      const T cn = sqrt(sh.res[2]);
      if (!(cn > 0)) break;
      const T inv = T(1) / cn;
      const T ar = sh.res[0] * inv, ai = sh.res[1] * inv;       // a_k = (chi_k, rho_k), chi_k = chi'_k / c_k
      if (threadIdx.x == 0) {
        sh.c[k] = cn;
        sh.a[2 * k] = ar;
        sh.a[2 * k + 1] = ai;
      }
      if (a.a3 && threadIdx.x < ns) {     // (chi_k, B^ g_l) = conj((B^ g_l, chi'_k)) / c_k
        sh.tg[k][2 * threadIdx.x] = sh.res[3 + 2 * threadIdx.x] * inv;
        sh.tg[k][2 * threadIdx.x + 1] = -sh.res[3 + 2 * threadIdx.x + 1] * inv;
      }
      // rho_{k+1} = rho_k - (a_k / c_k) chi'_k on this CTA's rows, into the other buffer
      const cplx<T> ack = {ar * inv, ai * inv};
      s1[0] = 0;
      cplx<T>* rn1 = rhob[cur ^ 1];
      slice([&](size_t i) {
        const cplx<T> y = rk[i] - ack * ck[i];
        rn1[i] = y;
        s1[0] += y.re * y.re + y.im * y.im;
      });
      cta_sum<T, 1>(sh, s1);
      if (threadIdx.x == 0) {
        sh.rr = sh.cta[0];
        sh.ac[0] = ack.re;
        sh.ac[1] = ack.im;
      }
      __syncthreads();
      cur ^= 1;
      ++total;
      // |rho_{k+1}|^2 = |rho_k|^2 - |a_k|^2 (one step of the recursion from the exact |rho_k|^2)
      const T est = rn2 - (ar * ar + ai * ai);
      rn = est > 0 ? sqrt(est) : T(0);
      if ((double)rn <= a.tol * (double)bn) { ++k; break; }
    }
    // back substitution by warp 0 (lane i holds row i), then v += sum beta_k xi_k
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      T br = lane < k ? sh.a[2 * lane] : T(0), bi = lane < k ? sh.a[2 * lane + 1] : T(0);
      for (int j = k - 1; j >= 0; --j) {
        const T cj = sh.c[j];
        const T yr = __shfl_sync(0xffffffffu, br, j) / cj, yi = __shfl_sync(0xffffffffu, bi, j) / cj;
        if (lane == j) { sh.beta[2 * j] = yr; sh.beta[2 * j + 1] = yi; }
        if (lane < j) {     // row lane -= bb[lane][j] beta_j
          const T mr = sh.bb[lane][2 * j], mi = sh.bb[lane][2 * j + 1];
          br -= mr * yr - mi * yi;
          bi -= mr * yi + mi * yr;
        }
      }
    }
    __syncthreads();
    slice([&](size_t i) {
      cplx<T> x = v[i];
#pragma unroll
      for (int j = 0; j < COOP_NKV; ++j)
        if (j < k) x += cplx<T>{sh.beta[2 * j], sh.beta[2 * j + 1]} * xi(j)[i];
      v[i] = x;
    });
    grid.sync();
    if (k == 0) break;
    // true residual of the deflated system
    coop_bhat<T, NS, RING>(grid, rg, a, v, tmpo, t, hp);
    if (a.a3) coop_PL<T, NS>(grid, sh, a, t, g, Bg, nullptr, sl);
    s1[0] = 0;
    cplx<T>* r0 = rhob[cur];
    slice([&](size_t i) {
      const cplx<T> y = rhsd[i] - t[i];
      r0[i] = y;
      s1[0] += y.re * y.re + y.im * y.im;
    });
    cta_sum<T, 1>(sh, s1);
    if (threadIdx.x == 0) sh.rr = sh.cta[0];
    coop_reduce(grid, sh, 1, a.acc);
    rn = sqrt(sh.res[0]);
  }
  if (a.a3) {
    // v = chi + g A~^{-1} g^+ (b - B^ chi)
    grid.sync();
    coop_bhat<T, NS, RING>(grid, rg, a, v, tmpo, t, hp);
    slice([&](size_t i) { t[i] = b[i] - t[i]; });
    coop_PL<T, NS>(grid, sh, a, t, g, g, v, sl);     // v += g z,  z = A~^{-1} g^+ t
  }
  if constexpr (RING) {
    // rows issued ahead for a hop that does not come: wait for their copies before exiting
    for (uint32_t q = rg.cons; q < rg.prod; ++q) mbar_wait(&rg.full[q % RING_SLOTS], (q / RING_SLOTS) & 1, rg.err);
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = total;
    a.out[1] = bn > 0 ? (double)rn / (double)bn : 0.0;
    if (RING && *(volatile int*)a.err) a.out[1] = __longlong_as_double(0x7ff8000000000000LL);   // NaN: failed
  }
}

// ------------------------------------------------------------------ multi-RHS cooperative little GCR
// Up to COOP_MAXR little systems with the same operator, solved in lockstep by one persistent kernel
// (FP32).  The GCR steps of all systems share the hops (each operator block is read once per step
// for all of them), the grid barriers and the reductions; every system keeps its own scalars,
// tolerance and convergence flag and is frozen once it has converged.  A step is the one of the
// one-system kernel: odd hop on rho_{k-1} - (a/c) chi'_{k-1}, even hop, one reduction for g^+ chi_k,
// (chi'_j, chi_k) and |rho_k|^2, the projected and orthogonalised chi'_k with its inner products, a
// second reduction, the local update of rho.  The vectors hold the systems innermost, padded to RP
// (a power of two, >= 2): entry i of system r at [i RP + r], padding entries zero.  In the passes
// over a CTA's entries a lane always serves the same pair of systems (one float4) and every entry
// is always handled by the same thread, so the per-system sums meet by warp shuffles and the passes
// need no CTA barrier between them; the sums over CTAs are FP64 atomics, one grid barrier each.
constexpr int COOP_MAXR = 12;
constexpr int COOP_MRP = 16;                              // RP of COOP_MAXR systems
constexpr int COOP_MST = 2 * 32 + 2 * COOP_NKV + 4;       // reduced values per system, at most
constexpr int COOP_MNV = COOP_MAXR * COOP_MST;
constexpr int COOP_MVG = 8;                               // vectors per pass of the slice inner products

DW_HD int coop_mrp(int R) {
  int p = 2;
  while (p < R) p <<= 1;
  return p;
}

struct CoopMArgs {
  int Ne, No, nkv, maxit, a3, R, RP;
  const int *list_e, *list_o, *lnb_e, *lnb_o;
  const float *M, *g, *Bg, *Ainv;
  const float* b;     // [R][Ne Ns] complex right-hand sides
  const float* tol;   // [R] relative tolerances
  float* v;           // [R][Ne Ns] complex solutions
  float* work;        // 2 nkv + 6 vectors of max(Ne, No) Ns RP complex
  float* scratch;     // per-CTA coefficient tables, coop_m_cta_scratch(Ns) floats each
  double* acc;        // [3][COOP_MNV] reduction accumulators, zero at launch
  double* out;        // [R][2]: iterations, relative residual
};

struct __align__(16) CoopMShared {
  float cta[COOP_MNV];                                   // this CTA's share of a reduction
  float res[COOP_MNV];                                   // the reduced values
  float part[COOP_WARPS][COOP_MVG][COOP_MRP / 2][4];     // warp sums of the slice inner products
  float ainv[2 * 32 * 32];                               // A~^{-1}, row-major
  float z[32][COOP_MRP][2];                              // A~^{-1} u per system (zero for idle ones)
  float bbn[COOP_NKV][COOP_MRP][2];                      // coefficients on chi'_j of a slice update
  float cf[COOP_MRP][2];                                 // a_k / c_k of the current step
  float ac[COOP_MRP][2];                                 // a_{k-1} / c_{k-1}: rho_k = rho_{k-1} - ac chi'_{k-1}
  float rr[COOP_MRP];                                    // this CTA's share of |rho_k|^2 (next reduction)
  float c[COOP_MAXR][COOP_NKV], a[COOP_MAXR][2 * COOP_NKV], beta[COOP_MAXR][2 * COOP_NKV];
  float bn[COOP_MAXR], rn[COOP_MAXR], rn2[COOP_MAXR];
  int live[COOP_MAXR], kr[COOP_MAXR], its[COOP_MAXR];
  int phase, any;
};

// dynamic shared memory: the operator blocks of a row Ms [2][8 NS NS] and the staged neighbour
// blocks xs, cs [2][8 NS RP] (double-buffered), direction sums hp [8][NS RP], complex
__host__ __device__ inline size_t coop_m_dyn_bytes(int ns, int rp) {
  return ((size_t)2 * 8 * ns * ns + (size_t)2 * 2 * 8 * ns * rp + (size_t)8 * ns * rp) * 2 * sizeof(float);
}
// per-CTA global scratch of the multi-RHS solver: tg [COOP_MAXR][COOP_NKV][NS] = (chi_j, B^ g_l) and
// the GCR coefficients bb [COOP_MAXR][COOP_NKV][COOP_NKV], complex
__host__ __device__ inline size_t coop_m_cta_scratch(int ns) {
  return (size_t)COOP_MAXR * COOP_NKV * (ns + COOP_NKV) * 2;          // floats
}

DW_D void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
DW_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
DW_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// sums of sh.cta[0..nv) over all CTAs into sh.res: FP64 atomics into accumulator set (phase mod 3),
// one grid barrier; CTA 0 clears the set used two reductions ahead (as coop_reduce)
DW_D void coop_mreduce(cg::grid_group& grid, CoopMShared& sh, int nv, double* acc_base) {
  __syncthreads();
  double* acc = acc_base + (size_t)(sh.phase % 3) * COOP_MNV;
  for (int v = threadIdx.x; v < nv; v += COOP_THREADS) atomicAdd(acc + v, (double)sh.cta[v]);
  __syncthreads();
  grid.sync();
  for (int v = threadIdx.x; v < nv; v += COOP_THREADS) sh.res[v] = (float)__ldcg(acc + v);
  if (blockIdx.x == 0) {
    double* old = acc_base + (size_t)((sh.phase + 2) % 3) * COOP_MNV;
    for (int v = threadIdx.x; v < COOP_MNV; v += COOP_THREADS) old[v] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.phase += 1;
  __syncthreads();
}

// lane mapping of the passes over this CTA's even entries s0 + e, e < S: the thread handles the
// system pair rq (float4 rq of an entry, RP / 2 per entry) of the entries e0, e0 + estep, ...
template <int RP>
struct MLane {
  static constexpr int RQ = RP / 2, EPW = 32 / RQ, ESTEP = COOP_WARPS * EPW;
  int rq, e0, S;
  size_t s0;
  DW_D MLane(int nrow, int ns) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    rq = lane % RQ;
    e0 = w * EPW + lane / RQ;
    int rb, re;
    coop_row_range(nrow, &rb, &re);
    s0 = (size_t)rb * ns;
    S = (re - rb) * ns;
  }
};

// per-thread values s[h NV + f] (value f of system 2 rq + h) -> their CTA sums dst[r ST + off + f]
template <int RP, int NV>
DW_D void mslice_sum(CoopMShared& sh, const MLane<RP>& ml, float (&s)[2 * NV], int R, float* dst, int ST, int off) {
  constexpr int RQ = RP / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = RQ; o < 32; o <<= 1)
#pragma unroll
    for (int m = 0; m < 2 * NV; ++m) s[m] += __shfl_xor_sync(0xffffffffu, s[m], o);
  if (lane < RQ)
#pragma unroll
    for (int m = 0; m < 2 * NV; ++m) (&sh.part[w][0][0][0])[ml.rq * 2 * NV + m] = s[m];
  __syncthreads();
  for (int t = threadIdx.x; t < RQ * 2 * NV; t += COOP_THREADS) {
    const int q = t / (2 * NV), m = t - q * 2 * NV, h = m / NV, f = m - h * NV, r = 2 * q + h;
    if (r < R) {
      float x = 0.f;
#pragma unroll
      for (int ww = 0; ww < COOP_WARPS; ++ww) x += (&sh.part[ww][0][0][0])[t];
      dst[r * ST + off + f] = x;
    }
  }
  __syncthreads();
}

// sh.cta[r ST + off + 2v (+1)] = this CTA's share of (X_v, Y_r), v < nvec, r < R.  SHX: X_v is one
// vector for all systems (entry i at X_v[i], vectors xs complex apart); otherwise X_v holds all
// systems like Y (vectors xs complex apart).
template <int RP, bool SHX>
DW_D void mslice_dots(CoopMShared& sh, const MLane<RP>& ml, const float* X, size_t xs, int nvec, const float* Y, int R,
                      int ST, int off) {
  constexpr int RQ = RP / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float4* Y4 = reinterpret_cast<const float4*>(Y);
  for (int v0 = 0; v0 < nvec; v0 += COOP_MVG) {
    float acc[COOP_MVG][4];
#pragma unroll
    for (int u = 0; u < COOP_MVG; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
    // two entries per pass: the loads of both are in flight together
    constexpr int ES = MLane<RP>::ESTEP;
    for (int e = ml.e0; e < ml.S; e += 2 * ES) {
      const bool two = e + ES < ml.S;
      const size_t i0 = ml.s0 + e, i1 = two ? i0 + ES : i0;
      const float4 ya = __ldcg(Y4 + i0 * RQ + ml.rq);
      float4 yb = __ldcg(Y4 + i1 * RQ + ml.rq);
      if (!two) yb = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < COOP_MVG; ++u) {
        if (v0 + u < nvec) {
          if constexpr (SHX) {
            const float2* Xv = reinterpret_cast<const float2*>(X) + (size_t)(v0 + u) * xs;
            const float2 p = __ldg(Xv + i0), pb = __ldg(Xv + i1);
            acc[u][0] = fmaf(pb.y, yb.y, fmaf(pb.x, yb.x, fmaf(p.y, ya.y, fmaf(p.x, ya.x, acc[u][0]))));
            acc[u][1] = fmaf(-pb.y, yb.x, fmaf(pb.x, yb.y, fmaf(-p.y, ya.x, fmaf(p.x, ya.y, acc[u][1]))));
            acc[u][2] = fmaf(pb.y, yb.w, fmaf(pb.x, yb.z, fmaf(p.y, ya.w, fmaf(p.x, ya.z, acc[u][2]))));
            acc[u][3] = fmaf(-pb.y, yb.z, fmaf(pb.x, yb.w, fmaf(-p.y, ya.z, fmaf(p.x, ya.w, acc[u][3]))));
          } else {
            const float4* Xv = reinterpret_cast<const float4*>(X + 2 * (size_t)(v0 + u) * xs) + ml.rq;
            const float4 p = __ldcg(Xv + i0 * RQ), pb = __ldcg(Xv + i1 * RQ);
            acc[u][0] = fmaf(pb.y, yb.y, fmaf(pb.x, yb.x, fmaf(p.y, ya.y, fmaf(p.x, ya.x, acc[u][0]))));
            acc[u][1] = fmaf(-pb.y, yb.x, fmaf(pb.x, yb.y, fmaf(-p.y, ya.x, fmaf(p.x, ya.y, acc[u][1]))));
            acc[u][2] = fmaf(pb.w, yb.w, fmaf(pb.z, yb.z, fmaf(p.w, ya.w, fmaf(p.z, ya.z, acc[u][2]))));
            acc[u][3] = fmaf(-pb.w, yb.z, fmaf(pb.z, yb.w, fmaf(-p.w, ya.z, fmaf(p.z, ya.w, acc[u][3]))));
          }
        }
      }
    }
#pragma unroll
    for (int o = RQ; o < 32; o <<= 1)
#pragma unroll
      for (int u = 0; u < COOP_MVG; ++u)
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[u][m] += __shfl_xor_sync(0xffffffffu, acc[u][m], o);
    if (lane < RQ)
#pragma unroll
      for (int u = 0; u < COOP_MVG; ++u)
#pragma unroll
        for (int m = 0; m < 4; ++m) sh.part[w][u][ml.rq][m] = acc[u][m];
    __syncthreads();
    for (int t = threadIdx.x; t < COOP_MVG * RQ * 4; t += COOP_THREADS) {
      const int u = t / (RQ * 4), q = (t >> 2) % RQ, m = t & 3, r = 2 * q + (m >> 1);
      if (v0 + u < nvec && r < R) {
        float x = 0.f;
#pragma unroll
        for (int ww = 0; ww < COOP_WARPS; ++ww) x += sh.part[ww][u][q][m];
        sh.cta[r * ST + off + 2 * (v0 + u) + (m & 1)] = x;
      }
    }
    __syncthreads();
  }
}

// out = base + sign * sum_d M[list[row]][d] src[lnb[row][d]] on this CTA's rows, all systems (vectors
// with RP systems innermost); with corr the source is src - ac_r corr (ac from sh).  The operator
// blocks of a row and its 8 neighbour blocks are copied into shared memory by cp.async one row
// ahead (double buffers); warp d multiplies block d, lane k holding the column entries M(k, c) in
// registers, into all systems (four independent FMA chains per system pair); the direction sums
// meet in shared memory.
template <int NS, int RP>
DW_D void coop_mhop(int nrow, int R, const int* list, const int* lnb, const float* M, const float* src,
                    const float* corr, const CoopMShared& sh, const float* base, float* out, float sign,
                    float4* Ms, float4* xs, float4* cs, float4* hp) {
  constexpr int RQ = RP / 2, BLK4 = NS * RQ, NST = 8 * BLK4;          // float4 of a row's neighbour data
  constexpr int MB4 = 8 * NS * NS / 2;                                  // float4 of a row's operator blocks
  constexpr int QG = 32 / NS;                                           // lane groups (system pairs split)
  static_assert(NS % 2 == 0 && NS <= 32, "even Ns <= 32");
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kk = lane % NS, q = lane / NS;
  const float4* S4 = reinterpret_cast<const float4*>(src);
  const float4* C4 = reinterpret_cast<const float4*>(corr);
  int rb, re;
  coop_row_range(nrow, &rb, &re);
  auto issue = [&](int row, int buf) {
    const float4* Mg = reinterpret_cast<const float4*>(M) + (size_t)__ldg(list + row) * MB4;
    for (int t = threadIdx.x; t < MB4; t += COOP_THREADS) cp_async16(Ms + buf * MB4 + t, Mg + t);
    for (int t = threadIdx.x; t < NST; t += COOP_THREADS) {
      const int d = t / BLK4, o = t - d * BLK4;
      const size_t g4 = (size_t)__ldg(lnb + row * 8 + d) * BLK4 + o;
      cp_async16(xs + buf * NST + t, S4 + g4);
      if (corr) cp_async16(cs + buf * NST + t, C4 + g4);
    }
    cp_async_commit();
  };
  if (rb < re) issue(rb, 0);
  int buf = 0;
  for (int row = rb; row < re; ++row, buf ^= 1) {
    if (row + 1 < re) {
      issue(row + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    if (corr)     // the elements this thread copied: x = src - ac corr
      for (int t = threadIdx.x; t < NST; t += COOP_THREADS) {
        const int r0 = 2 * (t % RQ);
        float4 x = xs[buf * NST + t];
        const float4 y = cs[buf * NST + t];
        const float c0r = sh.ac[r0][0], c0i = sh.ac[r0][1], c1r = sh.ac[r0 + 1][0], c1i = sh.ac[r0 + 1][1];
        x.x -= c0r * y.x - c0i * y.y;
        x.y -= c0r * y.y + c0i * y.x;
        x.z -= c1r * y.z - c1i * y.w;
        x.w -= c1r * y.w + c1i * y.z;
        xs[buf * NST + t] = x;
      }
    __syncthreads();
    if (q < QG) {
      const float2* Mw = reinterpret_cast<const float2*>(Ms + buf * MB4) + w * NS * NS + kk;
      float2 m[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) m[c] = Mw[c * NS];
      const float4* xd = xs + buf * NST + w * BLK4;
      float2* hd = reinterpret_cast<float2*>(hp) + (w * NS + kk) * RP;
#pragma unroll
      for (int u2 = q; u2 < RQ; u2 += QG) {
        if (2 * u2 < R) {
          float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
#pragma unroll
          for (int c = 0; c < NS; ++c) {
            const float4 x = xd[c * RQ + u2];
            ar0 = fmaf(-m[c].y, x.y, fmaf(m[c].x, x.x, ar0));
            ai0 = fmaf(m[c].y, x.x, fmaf(m[c].x, x.y, ai0));
            ar1 = fmaf(-m[c].y, x.w, fmaf(m[c].x, x.z, ar1));
            ai1 = fmaf(m[c].y, x.z, fmaf(m[c].x, x.w, ai1));
          }
          hd[2 * u2] = make_float2(ar0, ai0);
          hd[2 * u2 + 1] = make_float2(ar1, ai1);
        }
      }
    }
    __syncthreads();
    for (int tt = threadIdx.x; tt < BLK4; tt += COOP_THREADS) {
      const int r0 = 2 * (tt % RQ);
      float4 s = hp[tt];
#pragma unroll
      for (int d = 1; d < 8; ++d) {
        const float4 h = hp[d * BLK4 + tt];
        s.x += h.x; s.y += h.y; s.z += h.z; s.w += h.w;
      }
      const size_t o = (size_t)row * BLK4 + tt;
      float4 val = base ? __ldcg(reinterpret_cast<const float4*>(base) + o) : make_float4(0.f, 0.f, 0.f, 0.f);
      val.x = fmaf(sign, s.x, val.x); val.y = fmaf(sign, s.y, val.y);
      val.z = fmaf(sign, s.z, val.z); val.w = fmaf(sign, s.w, val.w);
      if (r0 >= R) val.x = val.y = 0.f;                   // padding systems stay zero
      if (r0 + 1 >= R) val.z = val.w = 0.f;
      reinterpret_cast<float4*>(out)[o] = val;
    }
  }
  __syncthreads();
}

template <int NS, int RP>
__global__ void __launch_bounds__(COOP_THREADS, 1) little_gcr_coop_mrhs_kernel(CoopMArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ CoopMShared sh;
  extern __shared__ __align__(16) unsigned char coop_mdyn[];
  constexpr int RQ = RP / 2;
  const int R = a.R, nkv = a.nkv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* Ms = reinterpret_cast<float4*>(coop_mdyn);                  // [2][8 NS NS / 2]
  float4* xs = Ms + 2 * 8 * NS * NS / 2;                              // [2][8 NS RQ]
  float4* cs = xs + 2 * 8 * NS * RQ;                                  // [2][8 NS RQ]
  float4* hp = cs + 2 * 8 * NS * RQ;                                  // [8][NS RQ]
  cplx<float>* tg = reinterpret_cast<cplx<float>*>(a.scratch + blockIdx.x * coop_m_cta_scratch(NS));
  cplx<float>* bbm = tg + (size_t)COOP_MAXR * COOP_NKV * NS;         // [R][nkv][nkv]
  auto TG = [&](int r, int j, int l) -> cplx<float>& { return tg[((size_t)r * COOP_NKV + j) * NS + l]; };
  auto BB = [&](int r, int j, int k) -> cplx<float>& { return bbm[((size_t)r * COOP_NKV + j) * COOP_NKV + k]; };
  const size_t n = (size_t)a.Ne * NS;                                // entries of an even vector
  const size_t vlen = (size_t)max(a.Ne, a.No) * NS * RP;             // complex numbers per work vector
  const MLane<RP> ml(a.Ne, NS);
  const int na = a.a3 ? 2 * NS : 0;
  auto V = [&](int qv) { return a.work + 2 * (size_t)qv * vlen; };
  auto V4 = [&](float* p) { return reinterpret_cast<float4*>(p); };
  // work vectors: chi'_j (j < nkv, unnormalised, norms c_j), xi_j, rho (two buffers), tmpo, t, rhsd, v
  float* rhob[2] = {V(2 * nkv), V(2 * nkv + 1)};
  float* tmpo = V(2 * nkv + 2);
  float* t = V(2 * nkv + 3);
  float* rhsd = V(2 * nkv + 4);
  float* vv = V(2 * nkv + 5);
  const float2* g2 = reinterpret_cast<const float2*>(a.g);
  const float2* Bg2 = reinterpret_cast<const float2*>(a.Bg);
  const float2* b2 = reinterpret_cast<const float2*>(a.b);
  auto slice4 = [&](auto&& f) {
    for (int e = ml.e0; e < ml.S; e += MLane<RP>::ESTEP) f(((size_t)ml.s0 + e) * RQ + ml.rq, (size_t)ml.s0 + e);
  };
  auto update_any = [&]() {
    __syncthreads();
    if (threadIdx.x == 0) {
      int x = 0;
      for (int r = 0; r < R; ++r) x |= sh.live[r];
      sh.any = x;
    }
    __syncthreads();
    return sh.any != 0;
  };
  // z_r = A~^{-1} u_r, u_r at sh.res[r ST + off ..]; only_live: zero for frozen systems
  auto mzsolve = [&](int ST, int off, bool only_live) {
    for (int tt = threadIdx.x; tt < COOP_MRP * NS; tt += COOP_THREADS) {
      const int r = tt / NS, l = tt - r * NS;
      float zr = 0.f, zi = 0.f;
      if (r < R && (!only_live || sh.live[r])) {
        for (int qq = 0; qq < NS; ++qq) {
          const float mr = sh.ainv[2 * (l * NS + qq)], mi = sh.ainv[2 * (l * NS + qq) + 1];
          const float yr = sh.res[r * ST + off + 2 * qq], yi = sh.res[r * ST + off + 2 * qq + 1];
          zr += mr * yr - mi * yi;
          zi += mr * yi + mi * yr;
        }
      }
      sh.z[l][r][0] = zr;
      sh.z[l][r][1] = zi;
    }
    __syncthreads();
  };
  // upd -= sg sum_l z_l vecs_l with z = A~^{-1} g^+ dot, for every system (A.3)
  auto mproject = [&](const float* dot, float* upd, const float2* vecs, float sg) {
    mslice_dots<RP, true>(sh, ml, a.g, n, NS, dot, R, 2 * NS, 0);
    coop_mreduce(grid, sh, R * 2 * NS, a.acc);
    mzsolve(2 * NS, 0, false);
    slice4([&](size_t q4, size_t i) {
      float4 x = __ldcg(V4(upd) + q4);
#pragma unroll
      for (int l = 0; l < NS; ++l) {
        const float2 gv = __ldg(vecs + (size_t)l * n + i);
        const float4 zz = *reinterpret_cast<const float4*>(&sh.z[l][2 * ml.rq][0]);
        x.x -= sg * (zz.x * gv.x - zz.y * gv.y);
        x.y -= sg * (zz.x * gv.y + zz.y * gv.x);
        x.z -= sg * (zz.z * gv.x - zz.w * gv.y);
        x.w -= sg * (zz.z * gv.y + zz.w * gv.x);
      }
      V4(upd)[q4] = x;
    });
  };
  // the sums of s2 (|.|^2 of the two systems of a thread) into sh.cta[r] and sh.rr[r]
  auto norm_share = [&](float (&s2)[2]) {
    mslice_sum<RP, 1>(sh, ml, s2, R, sh.cta, 1, 0);
    if (threadIdx.x < R) sh.rr[threadIdx.x] = sh.cta[threadIdx.x];
  };

  if (a.a3)
    for (int tt = threadIdx.x; tt < NS * NS; tt += COOP_THREADS) {
      sh.ainv[2 * tt] = a.Ainv[2 * tt];
      sh.ainv[2 * tt + 1] = a.Ainv[2 * tt + 1];
    }
  for (int tt = threadIdx.x; tt < 32 * COOP_MRP * 2; tt += COOP_THREADS) (&sh.z[0][0][0])[tt] = 0.f;
  for (int tt = threadIdx.x; tt < COOP_NKV * COOP_MRP * 2; tt += COOP_THREADS) (&sh.bbn[0][0][0])[tt] = 0.f;
  if (threadIdx.x < COOP_MRP) {
    sh.ac[threadIdx.x][0] = sh.ac[threadIdx.x][1] = 0.f;
    sh.cf[threadIdx.x][0] = sh.cf[threadIdx.x][1] = 0.f;
    sh.rr[threadIdx.x] = 0.f;
  }
  if (threadIdx.x < COOP_MAXR) {
    sh.its[threadIdx.x] = 0;
    sh.kr[threadIdx.x] = 0;
    sh.live[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) sh.phase = 0;
  __syncthreads();

  // rhsd = P~_L b (systems innermost, padding zero), rho_0 = rhsd, v = 0
  slice4([&](size_t q4, size_t i) {
    const int r0 = 2 * ml.rq;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 < R) { const float2 y = b2[(size_t)r0 * n + i]; x.x = y.x; x.y = y.y; }
    if (r0 + 1 < R) { const float2 y = b2[(size_t)(r0 + 1) * n + i]; x.z = y.x; x.w = y.y; }
    V4(rhsd)[q4] = x;
    V4(vv)[q4] = make_float4(0.f, 0.f, 0.f, 0.f);
  });
  if (a.a3) mproject(rhsd, rhsd, Bg2, 1.f);
  {
    float s2[2] = {0.f, 0.f};
    slice4([&](size_t q4, size_t) {
      const float4 x = __ldcg(V4(rhsd) + q4);
      V4(rhob[0])[q4] = x;
      s2[0] += x.x * x.x + x.y * x.y;
      s2[1] += x.z * x.z + x.w * x.w;
    });
    norm_share(s2);
  }
  coop_mreduce(grid, sh, R, a.acc);
  if (threadIdx.x < R) {
    const int r = threadIdx.x;
    sh.bn[r] = sqrtf(sh.res[r]);
    sh.rn[r] = sh.bn[r];
    sh.live[r] = sh.bn[r] > 0.f && a.maxit > 0;
  }
  int cur = 0;                                            // rhob[cur] holds rho_k on this CTA's rows
  while (update_any()) {
    if (threadIdx.x < R) sh.kr[threadIdx.x] = 0;
    __syncthreads();
    for (int k = 0; k < nkv; ++k) {
      float* ck = V(k);
      float* rk = rhob[cur];
      // xi_k = rho_k; chi_k = B^ rho_k (the odd hop reads rho_k of other CTAs as rho_{k-1} - ac chi'_{k-1})
      slice4([&](size_t q4, size_t) { V4(V(nkv + k))[q4] = __ldcg(V4(rk) + q4); });
      coop_mhop<NS, RP>(a.No, R, a.list_o, a.lnb_o, a.M, k > 0 ? rhob[cur ^ 1] : rk, k > 0 ? V(k - 1) : nullptr, sh,
                    nullptr, tmpo, 1.f, Ms, xs, cs, hp);
      grid.sync();
      __syncthreads();
      coop_mhop<NS, RP>(a.Ne, R, a.list_e, a.lnb_e, a.M, tmpo, nullptr, sh, rk, ck, -1.f, Ms, xs, cs, hp);
      // one reduction: u = g^+ chi_k (A.3), (chi'_j, chi_k) for j < k, |rho_k|^2
      const int ST1 = na + 2 * k + 1;
      if (a.a3) mslice_dots<RP, true>(sh, ml, a.g, n, NS, ck, R, ST1, 0);
      if (k > 0) mslice_dots<RP, false>(sh, ml, a.work, vlen, k, ck, R, ST1, na);
      if (threadIdx.x < R) sh.cta[threadIdx.x * ST1 + na + 2 * k] = sh.rr[threadIdx.x];
      coop_mreduce(grid, sh, R * ST1, a.acc);
      if (threadIdx.x < R) {
        const int r = threadIdx.x;
        sh.rn2[r] = sh.res[r * ST1 + na + 2 * k];
        sh.rn[r] = sqrtf(sh.rn2[r]);
        if (sh.live[r] && (double)sh.rn[r] <= (double)a.tol[r] * (double)sh.bn[r]) sh.live[r] = 0;
      }
      if (!update_any()) break;                           // every rho_k converged: chi_k unused
      if (a.a3) mzsolve(ST1, 0, true);
      // coefficients of P~_L chi_k on the normalised chi_j: (chi'_j, chi_k) / c_j - sum_l z_l (chi_j, B^ g_l)
      for (int tt = threadIdx.x; tt < COOP_MRP * k; tt += COOP_THREADS) {
        const int r = tt / k, j = tt - r * k;
        float br = 0.f, bi = 0.f, ic = 0.f;
        if (r < R && sh.live[r]) {
          ic = 1.f / sh.c[r][j];
          br = sh.res[r * ST1 + na + 2 * j] * ic;
          bi = sh.res[r * ST1 + na + 2 * j + 1] * ic;
          if (a.a3)
            for (int l = 0; l < NS; ++l) {
              const float zr = sh.z[l][r][0], zi = sh.z[l][r][1];
              const cplx<float> tv = TG(r, j, l);
              br -= zr * tv.re - zi * tv.im;
              bi -= zr * tv.im + zi * tv.re;
            }
          BB(r, j, k) = cplx<float>{br, bi};
        }
        sh.bbn[j][r][0] = br * ic;
        sh.bbn[j][r][1] = bi * ic;
      }
      __syncthreads();
      // chi'_k = P~_L chi_k - sum_j b_jk chi'_j / c_j in place; (chi'_k, rho_k), |chi'_k|^2
      {
        float s6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        slice4([&](size_t q4, size_t i) {
          float4 y = __ldcg(V4(ck) + q4), y2 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (a.a3) {
#pragma unroll
            for (int l = 0; l < NS; ++l) {
              const float2 bg = __ldg(Bg2 + (size_t)l * n + i);
              const float4 zz = *reinterpret_cast<const float4*>(&sh.z[l][2 * ml.rq][0]);
              float4& u = (l & 1) ? y2 : y;
              u.x -= zz.x * bg.x - zz.y * bg.y;
              u.y -= zz.x * bg.y + zz.y * bg.x;
              u.z -= zz.z * bg.x - zz.w * bg.y;
              u.w -= zz.z * bg.y + zz.w * bg.x;
            }
          }
#pragma unroll
          for (int j = 0; j < COOP_NKV; ++j) {
            if (j < k) {
              const float4 x = __ldcg(V4(V(j)) + q4);
              const float4 bb = *reinterpret_cast<const float4*>(&sh.bbn[j][2 * ml.rq][0]);
              float4& u = (j & 1) ? y2 : y;
              u.x -= bb.x * x.x - bb.y * x.y;
              u.y -= bb.x * x.y + bb.y * x.x;
              u.z -= bb.z * x.z - bb.w * x.w;
              u.w -= bb.z * x.w + bb.w * x.z;
            }
          }
          y.x += y2.x; y.y += y2.y; y.z += y2.z; y.w += y2.w;
          V4(ck)[q4] = y;
          const float4 r = __ldcg(V4(rk) + q4);
          s6[0] += y.x * r.x + y.y * r.y;
          s6[1] += y.x * r.y - y.y * r.x;
          s6[2] += y.x * y.x + y.y * y.y;
          s6[3] += y.z * r.z + y.w * r.w;
          s6[4] += y.z * r.w - y.w * r.z;
          s6[5] += y.z * y.z + y.w * y.w;
        });
        const int ST2 = 3 + na;
        mslice_sum<RP, 3>(sh, ml, s6, R, sh.cta, ST2, 0);
        if (a.a3) mslice_dots<RP, true>(sh, ml, a.Bg, n, NS, ck, R, ST2, 3);
        coop_mreduce(grid, sh, R * ST2, a.acc);
        // per system: c_k = |chi'_k|, a_k = (chi_k, rho_k), the rho update coefficient a_k / c_k
        if (threadIdx.x < COOP_MRP) {
          const int r = threadIdx.x;
          float ar = 0.f, ai = 0.f, inv = 0.f;
          if (r < R && sh.live[r]) {
            const float cn = sqrtf(sh.res[r * ST2 + 2]);
            inv = cn > 0.f ? 1.f / cn : 0.f;
            ar = sh.res[r * ST2] * inv;
            ai = sh.res[r * ST2 + 1] * inv;
            if (cn > 0.f && ar == ar && ai == ai) {
              sh.c[r][k] = cn;
              sh.a[r][2 * k] = ar;
              sh.a[r][2 * k + 1] = ai;
            } else {                                      // breakdown: the cycle of r ends with k steps
              sh.live[r] = 0;
              ar = ai = inv = 0.f;
            }
          }
          sh.cf[r][0] = ar * inv;
          sh.cf[r][1] = ai * inv;
        }
        __syncthreads();
        if (a.a3)       // (chi_k, B^ g_l) = conj((B^ g_l, chi'_k)) / c_k
          for (int tt = threadIdx.x; tt < R * NS; tt += COOP_THREADS) {
            const int r = tt / NS, l = tt - r * NS;
            if (sh.live[r]) {
              const float inv = 1.f / sh.c[r][k];
              TG(r, k, l) = cplx<float>{sh.res[r * ST2 + 3 + 2 * l] * inv, -sh.res[r * ST2 + 3 + 2 * l + 1] * inv};
            }
          }
      }
      // rho_{k+1} = rho_k - (a_k / c_k) chi'_k on this CTA's rows, into the other buffer
      {
        float s2[2] = {0.f, 0.f};
        float* rn1 = rhob[cur ^ 1];
        slice4([&](size_t q4, size_t) {
          const float4 cf = *reinterpret_cast<const float4*>(&sh.cf[2 * ml.rq][0]);
          const float4 x = __ldcg(V4(ck) + q4), r = __ldcg(V4(rk) + q4);
          float4 y;
          y.x = r.x - (cf.x * x.x - cf.y * x.y);
          y.y = r.y - (cf.x * x.y + cf.y * x.x);
          y.z = r.z - (cf.z * x.z - cf.w * x.w);
          y.w = r.w - (cf.z * x.w + cf.w * x.z);
          V4(rn1)[q4] = y;
          s2[0] += y.x * y.x + y.y * y.y;
          s2[1] += y.z * y.z + y.w * y.w;
        });
        mslice_sum<RP, 1>(sh, ml, s2, R, sh.rr, 1, 0);
      }
      if (threadIdx.x < COOP_MRP) {
        const int r = threadIdx.x;
        sh.ac[r][0] = sh.cf[r][0];
        sh.ac[r][1] = sh.cf[r][1];
        if (r < R && sh.live[r]) {
          sh.its[r] += 1;
          sh.kr[r] = k + 1;
          // |rho_{k+1}|^2 = |rho_k|^2 - |a_k|^2: stop stepping this system once it is below the tolerance
          const float ar = sh.a[r][2 * k], ai = sh.a[r][2 * k + 1];
          const float est = sh.rn2[r] - (ar * ar + ai * ai);
          const float rne = est > 0.f ? sqrtf(est) : 0.f;
          if ((double)rne <= (double)a.tol[r] * (double)sh.bn[r] || sh.its[r] >= a.maxit) sh.live[r] = 0;
        }
      }
      cur ^= 1;
      if (!update_any()) break;
    }
    // back substitution per system (warp r), then v += sum_j beta_j xi_j
    __syncthreads();
    for (int r = w; r < R; r += COOP_WARPS) {
      const int kk = sh.kr[r];
      float br = lane < kk ? sh.a[r][2 * lane] : 0.f, bi = lane < kk ? sh.a[r][2 * lane + 1] : 0.f;
      for (int j = kk - 1; j >= 0; --j) {
        const float cj = sh.c[r][j];
        const float yr = __shfl_sync(0xffffffffu, br, j) / cj, yi = __shfl_sync(0xffffffffu, bi, j) / cj;
        if (lane == j) {
          sh.beta[r][2 * j] = yr;
          sh.beta[r][2 * j + 1] = yi;
        }
        if (lane < j) {
          const cplx<float> mv = BB(r, lane, j);
          br -= mv.re * yr - mv.im * yi;
          bi -= mv.re * yi + mv.im * yr;
        }
      }
    }
    __syncthreads();
    int kmax = 0;
    for (int r = 0; r < R; ++r) kmax = max(kmax, sh.kr[r]);
    for (int tt = threadIdx.x; tt < COOP_NKV * COOP_MRP; tt += COOP_THREADS) {
      const int j = tt / COOP_MRP, r = tt - j * COOP_MRP;
      const bool u = r < R && j < sh.kr[r];
      sh.bbn[j][r][0] = u ? sh.beta[r][2 * j] : 0.f;
      sh.bbn[j][r][1] = u ? sh.beta[r][2 * j + 1] : 0.f;
    }
    __syncthreads();
    slice4([&](size_t q4, size_t) {
      float4 x = __ldcg(V4(vv) + q4);
#pragma unroll
      for (int j = 0; j < COOP_NKV; ++j) {
        if (j < kmax) {
          const float4 xx = __ldcg(V4(V(nkv + j)) + q4);
          const float4 bb = *reinterpret_cast<const float4*>(&sh.bbn[j][2 * ml.rq][0]);
          x.x += bb.x * xx.x - bb.y * xx.y;
          x.y += bb.x * xx.y + bb.y * xx.x;
          x.z += bb.z * xx.z - bb.w * xx.w;
          x.w += bb.z * xx.w + bb.w * xx.z;
        }
      }
      V4(vv)[q4] = x;
    });
    __syncthreads();
    grid.sync();
    if (kmax == 0) break;                                 // nothing changed since the last true residual
    // true residuals of the deflated systems: rho = P~_L (rhsd - B^ v)
    coop_mhop<NS, RP>(a.No, R, a.list_o, a.lnb_o, a.M, vv, nullptr, sh, nullptr, tmpo, 1.f, Ms, xs, cs, hp);
    grid.sync();
    __syncthreads();
    coop_mhop<NS, RP>(a.Ne, R, a.list_e, a.lnb_e, a.M, tmpo, nullptr, sh, vv, t, -1.f, Ms, xs, cs, hp);
    if (a.a3) mproject(t, t, Bg2, 1.f);
    {
      float s2[2] = {0.f, 0.f};
      float* r0p = rhob[cur];
      slice4([&](size_t q4, size_t) {
        const float4 x = __ldcg(V4(rhsd) + q4), tt4 = __ldcg(V4(t) + q4);
        const float4 y = make_float4(x.x - tt4.x, x.y - tt4.y, x.z - tt4.z, x.w - tt4.w);
        V4(r0p)[q4] = y;
        s2[0] += y.x * y.x + y.y * y.y;
        s2[1] += y.z * y.z + y.w * y.w;
      });
      norm_share(s2);
    }
    coop_mreduce(grid, sh, R, a.acc);
    if (threadIdx.x < R) {
      const int r = threadIdx.x;
      sh.rn[r] = sqrtf(sh.res[r]);
      sh.live[r] = sh.bn[r] > 0.f && (double)sh.rn[r] > (double)a.tol[r] * (double)sh.bn[r] && sh.its[r] < a.maxit;
    }
    if (threadIdx.x < COOP_MRP) sh.ac[threadIdx.x][0] = sh.ac[threadIdx.x][1] = 0.f;
  }
  if (a.a3) {
    // v = chi + g A~^{-1} g^+ (b - B^ chi) for every system
    grid.sync();
    __syncthreads();
    coop_mhop<NS, RP>(a.No, R, a.list_o, a.lnb_o, a.M, vv, nullptr, sh, nullptr, tmpo, 1.f, Ms, xs, cs, hp);
    grid.sync();
    __syncthreads();
    coop_mhop<NS, RP>(a.Ne, R, a.list_e, a.lnb_e, a.M, tmpo, nullptr, sh, vv, t, -1.f, Ms, xs, cs, hp);
    slice4([&](size_t q4, size_t i) {
      const int r0 = 2 * ml.rq;
      float4 x = __ldcg(V4(t) + q4);
      float4 bx = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 < R) { const float2 y = b2[(size_t)r0 * n + i]; bx.x = y.x; bx.y = y.y; }
      if (r0 + 1 < R) { const float2 y = b2[(size_t)(r0 + 1) * n + i]; bx.z = y.x; bx.w = y.y; }
      V4(t)[q4] = make_float4(bx.x - x.x, bx.y - x.y, bx.z - x.z, bx.w - x.w);
    });
    mproject(t, vv, g2, -1.f);
  }
  // the solutions in the [R][Ne Ns] layout
  slice4([&](size_t q4, size_t i) {
    const int r0 = 2 * ml.rq;
    const float4 x = __ldcg(V4(vv) + q4);
    float2* vo = reinterpret_cast<float2*>(a.v);
    if (r0 < R) vo[(size_t)r0 * n + i] = make_float2(x.x, x.y);
    if (r0 + 1 < R) vo[(size_t)(r0 + 1) * n + i] = make_float2(x.z, x.w);
  });
  if (blockIdx.x == 0 && threadIdx.x < R) {
    const int r = threadIdx.x;
    a.out[2 * r] = sh.its[r];
    a.out[2 * r + 1] = sh.bn[r] > 0.f ? (double)sh.rn[r] / (double)sh.bn[r] : 0.0;
  }
}

// ====================================================================== host side
template <typename T>
static const T* Mp(dfl_ctx* d);
template <> const float* Mp<float>(dfl_ctx* d) { return d->M32; }
template <> const double* Mp<double>(dfl_ctx* d) { return d->M64; }
template <typename T>
static const T* Binvp(dfl_ctx* d);
template <> const float* Binvp<float>(dfl_ctx* d) { return d->Binv32; }
template <> const double* Binvp<double>(dfl_ctx* d) { return d->Binv64; }
template <typename T>
static const T* gp(dfl_ctx* d);
template <> const float* gp<float>(dfl_ctx* d) { return d->g32; }
template <> const double* gp<double>(dfl_ctx* d) { return d->g64; }
template <typename T>
static const T* Bgp(dfl_ctx* d);
template <> const float* Bgp<float>(dfl_ctx* d) { return d->Bg32; }
template <> const double* Bgp<double>(dfl_ctx* d) { return d->Bg64; }

// B^ v_e = v_e - M_eo (M_oe v_e);  tmp_o: No*Ns complex
template <typename T>
static void apply_bhat(dfl_ctx* d, const T* ve, T* tmp_o, T* out, cudaStream_t s) {
  NS_DISPATCH(d->Ns, (little_hop_kernel<T, NSV><<<d->No, 256, 0, s>>>(
                                d->No, d->Ns, d->d_list[1], d->d_lnb[1], Mp<T>(d), ve, nullptr, tmp_o)));
  dw_note_launch();
  // tmp_o = -M_oe v_e; out = v_e - M_eo(M_oe v_e) = v_e + M_eo tmp_o  ->  use base = v_e and src = -tmp
  NS_DISPATCH(d->Ns, (little_hop_kernel<T, NSV><<<d->Ne, 256, 0, s>>>(
                                d->Ne, d->Ns, d->d_list[0], d->d_lnb[0], Mp<T>(d), tmp_o, nullptr, out)));
  dw_note_launch();
  // out = -M_eo tmp_o = M_eo M_oe v_e ; final = v_e - out
  blas_xpby<T>(ve, out, -1.0, 0.0, (size_t)d->Ne * d->Ns, s);
}

extern "C" int dfl_dims(const dfl_ctx* d, int* Nb, int* Ns) {
  if (!d) { dw_set_error("dfl_dims: null context"); return DW_EINVAL; }
  if (Nb) *Nb = d->Nb;
  if (Ns) *Ns = d->Ns;
  return DW_OK;
}

extern "C" void dfl_destroy(dfl_ctx* d) {
  if (!d) return;
  void* ptrs[] = {d->d_sub, d->d_sap2dfl, d->d_bnb, d->d_list[0], d->d_list[1], d->d_lnb[0], d->d_lnb[1],
                  d->basis64, d->basis16, d->B64, d->Binv64, d->Binv32, d->M64, d->M32, d->g64, d->g32,
                  d->Bg64, d->Bg32, d->lw[0], d->lw[1], d->B32, d->fw[0], d->fw[1], d->Ainv64, d->Ainv32,
                  d->coop_partial, d->coop_out, d->coop_err, d->ref64, d->ref32, d->ddf, d->ddl, d->mw, d->mio,
                  d->meo, d->macc, d->mscr, d->mtol, d->mout};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete d;
}

template <typename T, int NS>
static bool launch_restrict_ns(dfl_ctx* d, const T* psi, T* c, int nrhs, cudaStream_t s) {
  if constexpr (NS == 0 || !std::is_same<T, float>::value) {
    return false;
  } else {
    restrict_ns_kernel<T, NS><<<d->Nb, 128, 0, s>>>(d->c->g, d->d_sub, d->nsub, d->basis16 ? nullptr : d->basis64,
                                                    d->basis16, psi, c, nrhs, (size_t)d->c->V * 24,
                                                    (size_t)d->N * 2);
    return true;
  }
}
template <typename T>
static int restrict_t(dfl_ctx* d, const T* psi, T* c, cudaStream_t s, int nrhs = 1) {
  if (sizeof(T) == 4) {
    bool done = false;
    NS_DISPATCH(d->Ns, (done = launch_restrict_ns<T, NSV>(d, psi, c, nrhs, s)));
    if (done) { dw_note_launch(); return DW_OK; }
  }
  restrict_kernel<T><<<d->Nb, 128, 0, s>>>(d->c->g, d->d_sub, d->nsub, d->Ns, d->basis16 ? nullptr : d->basis64,
                                            d->basis16, psi, c, nrhs, (size_t)d->c->V * 24,
                                            (size_t)d->N * 2); dw_note_launch();
  return DW_OK;
}
template <typename T>
static int prolong_t(dfl_ctx* d, const T* c, T* psi, int mode, cudaStream_t s, int nrhs = 1) {
  unsigned blocks = (unsigned)((d->c->V + 127) / 128);
  prolong_kernel<T><<<blocks, 128, 0, s>>>(d->c->g, d->d_sap2dfl, d->Ns, d->basis16 ? nullptr : d->basis64,
                                            d->basis16, c, psi, mode, nrhs, (size_t)d->c->V * 24,
                                            (size_t)d->N * 2); dw_note_launch();
  return DW_OK;
}
// s + e += f x for an FP32 number f and a double-float x: the product split exactly into
// h + l (h = fl(f x.hi), its rounding error by one FMA, plus f x.lo), h added to s by TwoSum, the
// addition error and l added to the compensation e (compensated dot product, Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005)
DW_D void dot2_acc(float& s, float& e, float f, dd x) {
  const float h = __fmul_rn(f, x.hi);
  const float l = __fmaf_rn(f, x.lo, __fmaf_rn(f, x.hi, -h));
  const float t = __fadd_rn(s, h);
  const float b = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, b)), __fsub_rn(h, b));
  s = t;
  e = __fadd_rn(e, __fadd_rn(err, l));
}

// c[L][k] = (phi^L_k, psi) for a double-float psi and the BF16 basis (its entries are exact FP32
// numbers): per thread a compensated dot product (dot2_acc: about 11 FP32 operations per real
// product, against about 30 for full double-float arithmetic), then the threads' s + e combined
// in double-float arithmetic.  The result carries about twice the FP32 precision.  The Ns basis
// vectors are split over KG thread groups (warp-uniform), so each thread keeps 2 Ns / KG sums and
// the CTA has KG times the threads in flight on the basis loads.
template <int NS, int KG>
__global__ void __launch_bounds__(128 * KG) restrict_dd_bf16_kernel(Geom g, const int* __restrict__ sub, int nsub,
                                                                   const uint4* __restrict__ b16,
                                                                   const dd* __restrict__ psi0, dd* __restrict__ c0,
                                                                   int nrhs, size_t fstride, size_t cstride) {
  static_assert(NS % KG == 0, "the groups share the basis vectors evenly");
  constexpr int KP = NS / KG;                        // basis vectors per group
  using WH = WarpHalve<dd, 2 * KP, 16>;
  constexpr int MF = WH::final_m();
  __shared__ dd sh[4 * KG][2 * KP];
  const int L = blockIdx.x;
  const size_t V = g.V;
  const int nsite = nsub * g.svol;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = threadIdx.x >> 7, tl = threadIdx.x & 127, k0 = grp * KP;
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    const dd* psi = psi0 + (size_t)rhs * fstride;
    dd* c = c0 + (size_t)rhs * cstride;
    float sa[2 * KP], ea[2 * KP];
#pragma unroll
    for (int m = 0; m < 2 * KP; ++m) sa[m] = ea[m] = 0.f;
    for (int t = tl; t < nsite; t += 128) {
      const long long i = dfl_site(g, sub, nsub, L, t);
      cplx<dd> p[12];
      load_site<dd, 12>(psi, V, i, p);
#pragma unroll
      for (int kk = 0; kk < KP; ++kk) {
        cplx<float> f[12];
        load_basis<float>(nullptr, b16, V, k0 + kk, i, f);
#pragma unroll
        for (int j = 0; j < 12; ++j) {   // (f, p) = sum conj(f) p
          dot2_acc(sa[2 * kk], ea[2 * kk], f[j].re, p[j].re);
          dot2_acc(sa[2 * kk], ea[2 * kk], f[j].im, p[j].im);
          dot2_acc(sa[2 * kk + 1], ea[2 * kk + 1], f[j].re, p[j].im);
          dot2_acc(sa[2 * kk + 1], ea[2 * kk + 1], -f[j].im, p[j].re);
        }
      }
    }
    dd acc[2 * KP];
#pragma unroll
    for (int m = 0; m < 2 * KP; ++m) acc[m] = dd_two_sum(sa[m], ea[m]);
    int base = 0;
    WH::run(acc, lane, base);
#pragma unroll
    for (int m = 0; m < MF; ++m) sh[w][base + m] = acc[m];
    __syncthreads();
    if (tl < 2 * KP) {                 // warps 4 grp .. 4 grp + 3 hold group grp's sums
      dd y = sh[4 * grp][tl];
#pragma unroll
      for (int q = 1; q < 4; ++q) y += sh[4 * grp + q][tl];
      c[(size_t)L * 2 * NS + 2 * k0 + tl] = y;
    }
    __syncthreads();
  }
}

// psi = Phi c (the prolongation) for a double-float c and the BF16 basis: every output component a
// compensated sum (dot2_acc) of its 2 Ns products of an exact FP32 basis entry with a double-float
// coefficient; one thread per site.
template <int NS>
__global__ void __launch_bounds__(128) prolong_dd_bf16_kernel(Geom g, const int* __restrict__ sap2dfl,
                                                              const uint4* __restrict__ b16,
                                                              const dd* __restrict__ c, dd* __restrict__ psi) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  const size_t V = g.V;
  const int L = __ldg(sap2dfl + (int)(i >> g.lsvol));
  const cplx<dd>* cc = reinterpret_cast<const cplx<dd>*>(c) + (size_t)L * NS;
  float sa[24], ea[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) sa[m] = ea[m] = 0.f;
#pragma unroll 4
  for (int k = 0; k < NS; ++k) {
    const cplx<dd> ck = cc[k];
    cplx<float> f[12];
    load_basis<float>(nullptr, b16, V, k, i, f);
#pragma unroll
    for (int j = 0; j < 12; ++j) {   // ck f_j
      dot2_acc(sa[2 * j], ea[2 * j], f[j].re, ck.re);
      dot2_acc(sa[2 * j], ea[2 * j], -f[j].im, ck.im);
      dot2_acc(sa[2 * j + 1], ea[2 * j + 1], f[j].im, ck.re);
      dot2_acc(sa[2 * j + 1], ea[2 * j + 1], f[j].re, ck.im);
    }
  }
  cplx<dd> out[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) out[j] = {dd_two_sum(sa[2 * j], ea[2 * j]), dd_two_sum(sa[2 * j + 1], ea[2 * j + 1])};
  store_site<dd, 12>(psi, V, i, out);
}

// DW_DD_DOT2=0: full double-float arithmetic in the restriction (the compensated kernel's reference)
static bool dd_dot2_disabled() {
  const char* e = getenv("DW_DD_DOT2");
  return e && e[0] == '0';
}
template <int NS>
static bool launch_restrict_dd(dfl_ctx* d, const dd* psi, dd* c, cudaStream_t s) {
  if constexpr (NS == 0) {
    return false;
  } else {
    if (d->basis16 && !dd_dot2_disabled())
      restrict_dd_bf16_kernel<NS, (NS % 4 == 0 ? 4 : 2)><<<d->Nb, 128 * (NS % 4 == 0 ? 4 : 2), 0, s>>>(
          d->c->g, d->d_sub, d->nsub, d->basis16, psi, c, 1, (size_t)d->c->V * 24, (size_t)d->N * 2);
    else
      restrict_ns_kernel<dd, NS><<<d->Nb, 128, 0, s>>>(d->c->g, d->d_sub, d->nsub, d->basis16 ? nullptr : d->basis64,
                                                       d->basis16, psi, c, 1, (size_t)d->c->V * 24, (size_t)d->N * 2);
    return true;
  }
}
static int ensure_dd(dfl_ctx* d) {
  if (!d->ddf) DW_CUDA(cudaMalloc(&d->ddf, (size_t)d->c->V * 24 * sizeof(dd)));
  if (!d->ddl) DW_CUDA(cudaMalloc(&d->ddl, (size_t)d->N * 2 * sizeof(dd)));
  return DW_OK;
}
// c = Phi^+ psi for FP64 psi and c, computed in double-float arithmetic on the FP32 pipes
int dfl_restrict_f64x(dfl_ctx* d, const double* psi, double* c, cudaStream_t s) {
  int rc = ensure_dd(d);
  if (rc) return rc;
  f64_to_dd(psi, d->ddf, (size_t)d->c->V * 24, s);
  bool done = false;
  NS_DISPATCH_FEW(d->Ns, (done = launch_restrict_dd<NSV>(d, d->ddf, d->ddl, s)));
  if (!done)
    restrict_kernel<dd><<<d->Nb, 128, 0, s>>>(d->c->g, d->d_sub, d->nsub, d->Ns, d->basis16 ? nullptr : d->basis64,
                                              d->basis16, d->ddf, d->ddl, 1, (size_t)d->c->V * 24, (size_t)d->N * 2);
  dw_note_launch();
  dd_to_f64(d->ddl, c, (size_t)d->N * 2, 0, s);
  return DW_OK;
}
// psi = Phi c (add = 0) or psi += Phi c (add = 1), FP64 fields, double-float arithmetic
template <int NS>
static bool launch_prolong_dd(dfl_ctx* d, unsigned blocks, cudaStream_t s) {
  if constexpr (NS == 0) {
    return false;
  } else {
    prolong_dd_bf16_kernel<NS><<<blocks, 128, 0, s>>>(d->c->g, d->d_sap2dfl, d->basis16, d->ddl, d->ddf);
    return true;
  }
}
int dfl_prolong_f64x(dfl_ctx* d, const double* c, double* psi, int add, cudaStream_t s) {
  int rc = ensure_dd(d);
  if (rc) return rc;
  f64_to_dd(c, d->ddl, (size_t)d->N * 2, s);
  unsigned blocks = (unsigned)((d->c->V + 127) / 128);
  bool done = false;
  if (d->basis16 && !dd_dot2_disabled()) NS_DISPATCH_FEW(d->Ns, (done = launch_prolong_dd<NSV>(d, blocks, s)));
  if (!done)
    prolong_kernel<dd><<<blocks, 128, 0, s>>>(d->c->g, d->d_sap2dfl, d->Ns, d->basis16 ? nullptr : d->basis64,
                                              d->basis16, d->ddl, d->ddf, 0, 1, (size_t)d->c->V * 24,
                                              (size_t)d->N * 2);
  dw_note_launch();
  dd_to_f64(d->ddf, psi, (size_t)d->c->V * 24, add, s);
  return DW_OK;
}
int dfl_restrict_mrhs_f32(dfl_ctx* d, const float* psi, float* c, int nrhs, cudaStream_t s) {
  return restrict_t(d, psi, c, s, nrhs);
}
int dfl_prolong_mrhs_f32(dfl_ctx* d, const float* c, float* psi, int mode, int nrhs, cudaStream_t s) {
  return prolong_t(d, c, psi, mode, s, nrhs);
}
int dfl_restrict_f32(dfl_ctx* d, const float* psi, float* c, cudaStream_t s) { return restrict_t(d, psi, c, s); }
int dfl_restrict_f64(dfl_ctx* d, const double* psi, double* c, cudaStream_t s) { return restrict_t(d, psi, c, s); }
int dfl_prolong_f32(dfl_ctx* d, const float* c, float* psi, int mode, cudaStream_t s) {
  return prolong_t(d, c, psi, mode, s);
}
int dfl_prolong_f64(dfl_ctx* d, const double* c, double* psi, int mode, cudaStream_t s) {
  return prolong_t(d, c, psi, mode, s);
}

extern "C" int dfl_restrict(dfl_ctx* d, int prec, const void* psi, void* c, void* stream) {
  if (!d || !psi || !c || (prec != DW_F32 && prec != DW_F64 && prec != DW_F64X)) {
    dw_set_error("dfl_restrict: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == DW_F64X) {
    int rc = dfl_restrict_f64x(d, (const double*)psi, (double*)c, s);
    if (rc) return rc;
    DW_CUDA(cudaGetLastError());
    return DW_OK;
  }
  if (prec == DW_F64) restrict_t(d, (const double*)psi, (double*)c, s);
  else restrict_t(d, (const float*)psi, (float*)c, s);
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
extern "C" int dfl_prolong(dfl_ctx* d, int prec, const void* c, void* psi, void* stream) {
  if (!d || !psi || !c || (prec != DW_F32 && prec != DW_F64 && prec != DW_F64X)) {
    dw_set_error("dfl_prolong: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == DW_F64X) {
    int rc = dfl_prolong_f64x(d, (const double*)c, (double*)psi, 0, s);
    if (rc) return rc;
    DW_CUDA(cudaGetLastError());
    return DW_OK;
  }
  if (prec == DW_F64) prolong_t(d, (const double*)c, (double*)psi, 0, s);
  else prolong_t(d, (const float*)c, (float*)psi, 0, s);
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
extern "C" int dfl_basis_export(dfl_ctx* d, double* canon, void* stream) {
  if (!d || !canon) { dw_set_error("dfl_basis_export: bad argument"); return DW_EINVAL; }
  if (d->basis64) return dw_unpack(d->c, DW_F64, d->Ns, d->basis64, canon, stream);
  // BF16 basis: expand to FP64 in a temporary field block
  cudaStream_t s = (cudaStream_t)stream;
  const size_t V = d->c->V;
  double* tmp = nullptr;
  DW_CUDA(cudaMallocAsync((void**)&tmp, (size_t)d->Ns * 24 * V * sizeof(double), s));
  dequantize_kernel<<<(unsigned)((V * d->Ns + 255) / 256), 256, 0, s>>>(V, d->Ns, d->basis16, tmp); dw_note_launch();
  int rc = dw_unpack(d->c, DW_F64, d->Ns, tmp, canon, stream);
  cudaFreeAsync(tmp, s);
  return rc;
}

// A BF16 basis needs its FP64 expansion only while the little operator is assembled: drop it
// afterwards (the restriction and prolongation kernels read the BF16 basis).  Saves Ns FP64 fields.
static void drop_basis64(dfl_ctx* d) {
  if (d->basis16 && d->basis64) {
    cudaFree(d->basis64);
    d->basis64 = nullptr;
  }
}
extern "C" int little_apply(dfl_ctx* d, const double* v, double* w, void* stream) {
  if (!d || !v || !w || v == w) { dw_set_error("little_apply: bad argument"); return DW_EINVAL; }
  little_full_kernel<<<warps_grid(d->Nb), 128, 0, (cudaStream_t)stream>>>(d->Nb, d->Ns, d->d_bnb, d->B64, v, w); dw_note_launch();
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

// ---------------------------------------------------------------------- little GCR
// Work buffers (precision T), each n = Ne*Ns complex:
//   0..nkv-1 chi, nkv..2nkv-1 xi (= rho_k copies), then rho, t, tmp_o, wt, yo, ...
template <typename T>
static T* lwork(dfl_ctx* d, int idx) {
  constexpr int P = prec_of<T>();
  size_t n = (size_t)d->Ne * d->Ns * 2;
  return (T*)d->lw[P] + (size_t)idx * n;
}

static int sync_read(dw_ctx* c, const double* dev, int count, double* host, cudaStream_t s) {
  DW_CUDA(cudaMemcpyAsync(c->h_red, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) host[i] = c->h_red[i];
  return DW_OK;
}

// P~_L u (in place): u -= (B^ g) A~^{-1} g^+ u.  scratch: device double[2*Ns]
template <typename T>
static int little_PL(dfl_ctx* d, T* u, cudaStream_t s) {
  const int Ns = d->Ns;
  size_t n = (size_t)d->Ne * Ns;
  std::vector<const T*> gs(Ns), bgs(Ns);
  for (int l = 0; l < Ns; ++l) { gs[l] = gp<T>(d) + (size_t)l * 2 * n; bgs[l] = Bgp<T>(d) + (size_t)l * 2 * n; }
  double* dres = d->c->d_red + 65536;
  blas_multi_dot<T>(d->c, gs.data(), Ns, u, n, dres, s);
  std::vector<double> h(2 * Ns);
  int rc = sync_read(d->c, dres, 2 * Ns, h.data(), s);
  if (rc) return rc;
  std::vector<double> y(2 * Ns);
  for (int a = 0; a < Ns; ++a) {
    cd acc = 0;
    for (int b = 0; b < Ns; ++b) acc += d->Atil_inv[a * Ns + b] * cd(h[2 * b], h[2 * b + 1]);
    y[2 * a] = acc.real();
    y[2 * a + 1] = acc.imag();
  }
  blas_multi_axpy<T>(bgs.data(), Ns, y.data(), u, n, s);
  return DW_OK;
}

// v_e += g A~^{-1} g^+ r   (the coarse correction)
template <typename T>
static int little_coarse_add(dfl_ctx* d, const T* r, T* v, cudaStream_t s) {
  const int Ns = d->Ns;
  size_t n = (size_t)d->Ne * Ns;
  std::vector<const T*> gs(Ns);
  for (int l = 0; l < Ns; ++l) gs[l] = gp<T>(d) + (size_t)l * 2 * n;
  double* dres = d->c->d_red + 65536;
  blas_multi_dot<T>(d->c, gs.data(), Ns, r, n, dres, s);
  std::vector<double> h(2 * Ns);
  int rc = sync_read(d->c, dres, 2 * Ns, h.data(), s);
  if (rc) return rc;
  std::vector<double> y(2 * Ns);
  for (int a = 0; a < Ns; ++a) {
    cd acc = 0;
    for (int b = 0; b < Ns; ++b) acc += d->Atil_inv[a * Ns + b] * cd(h[2 * b], h[2 * b + 1]);
    y[2 * a] = -acc.real();        // multi_axpy subtracts
    y[2 * a + 1] = -acc.imag();
  }
  blas_multi_axpy<T>(gs.data(), Ns, y.data(), v, n, s);
  return DW_OK;
}

// Restarted GCR for op(v) = rhs on small (little) vectors of n complex numbers.
// work: 2*nkv + 3 vectors of n complex.  Stops at ||rhs - op v|| <= tol ||rhs||.
template <typename T, typename Op>
static int gcr_small(dw_ctx* c, Op op, const T* rhs, T* v, size_t n, T* work, double tol, int maxit, int nkv,
                     int* iters, double* relres, cudaStream_t s) {
  T* chi0 = work;
  T* xi0 = work + (size_t)nkv * 2 * n;
  T* rho = work + (size_t)2 * nkv * 2 * n;
  T* t = rho + 2 * n;
  auto chi = [&](int k) { return chi0 + (size_t)k * 2 * n; };
  auto xi = [&](int k) { return xi0 + (size_t)k * 2 * n; };
  double* dres = c->d_red + 65536;
  std::vector<double> hbuf(2 * (nkv + 2));
  int rc;
  blas_dot<T>(c, rhs, rhs, n, dres, s);
  if ((rc = sync_read(c, dres, 3, hbuf.data(), s))) return rc;
  const double bn = sqrt(hbuf[2]);
  DW_CUDA(cudaMemsetAsync(v, 0, n * 2 * sizeof(T), s));
  *iters = 0;
  *relres = 0;
  if (bn == 0.0) return DW_OK;
  DW_CUDA(cudaMemcpyAsync(rho, rhs, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s));
  double rn = bn;
  int total = 0;
  std::vector<cd> a(nkv), cc(nkv);
  std::vector<cd> bb((size_t)nkv * nkv);
  while (rn > tol * bn && total < maxit) {
    int k = 0;
    for (; k < nkv && total < maxit; ++k, ++total) {
      DW_CUDA(cudaMemcpyAsync(xi(k), rho, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s));
      if ((rc = op(xi(k), chi(k)))) return rc;
      if (k > 0) {
        std::vector<const T*> prev(k);
        for (int j = 0; j < k; ++j) prev[j] = chi(j);
        blas_multi_dot<T>(c, prev.data(), k, chi(k), n, dres, s);
        if ((rc = sync_read(c, dres, 2 * k, hbuf.data(), s))) return rc;
        for (int j = 0; j < k; ++j) bb[(size_t)j * nkv + k] = cd(hbuf[2 * j], hbuf[2 * j + 1]);
        blas_multi_axpy<T>(prev.data(), k, hbuf.data(), chi(k), n, s);
      }
      blas_dot<T>(c, chi(k), rho, n, dres, s);
      if ((rc = sync_read(c, dres, 3, hbuf.data(), s))) return rc;
      double ck = sqrt(hbuf[2]);
      if (!(ck > 0)) break;
      cc[k] = ck;
      a[k] = cd(hbuf[0], hbuf[1]) / ck;
      blas_scale<T>(chi(k), 1.0 / ck, 0.0, n, s);
      blas_axpy<T>(chi(k), rho, -a[k].real(), -a[k].imag(), n, s);
      blas_dot<T>(c, rho, rho, n, dres, s);
      if ((rc = sync_read(c, dres, 3, hbuf.data(), s))) return rc;
      rn = sqrt(hbuf[2]);
      if (rn <= tol * bn) { ++k; ++total; break; }
    }
    std::vector<cd> beta(k);
    for (int j = k - 1; j >= 0; --j) {
      cd sacc = a[j];
      for (int i = j + 1; i < k; ++i) sacc -= bb[(size_t)j * nkv + i] * beta[i];
      beta[j] = sacc / cc[j];
    }
    std::vector<const T*> xs(k);
    std::vector<double> coef(2 * k);
    for (int j = 0; j < k; ++j) { xs[j] = xi(j); coef[2 * j] = -beta[j].real(); coef[2 * j + 1] = -beta[j].imag(); }
    if (k > 0) blas_multi_axpy<T>(xs.data(), k, coef.data(), v, n, s);
    if (k == 0) break;
    // true residual rho = rhs - op v
    if ((rc = op(v, t))) return rc;
    DW_CUDA(cudaMemcpyAsync(rho, rhs, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    blas_axpy<T>(t, rho, -1.0, 0.0, n, s);
    blas_dot<T>(c, rho, rho, n, dres, s);
    if ((rc = sync_read(c, dres, 3, hbuf.data(), s))) return rc;
    rn = sqrt(hbuf[2]);
  }
  *iters = total;
  *relres = rn / bn;
  return rn <= tol * bn ? DW_OK : DW_ENOTCONV;
}

template <typename T>
static const T* Ainvp(dfl_ctx* d);
template <> const float* Ainvp<float>(dfl_ctx* d) { return d->Ainv32; }
template <> const double* Ainvp<double>(dfl_ctx* d) { return d->Ainv64; }

static bool coop_enabled() {
  const char* e = getenv("DW_LITTLE_COOP");
  return !(e && e[0] == '0');
}

// the cooperative solver: same algorithm as little_gcr below (GCR on P~_L B^, then the A.3 correction)
template <typename T>
static int little_gcr_coop(dfl_ctx* d, const T* b, T* v, double tol, int maxit, int nkv, int* iters,
                           double* relres, cudaStream_t s) {
  CoopArgs<T> a;
  a.Ne = d->Ne; a.No = d->No; a.Ns = d->Ns; a.nkv = nkv; a.maxit = maxit; a.a3 = d->a3 ? 1 : 0;
  a.list_e = d->d_list[0]; a.list_o = d->d_list[1]; a.lnb_e = d->d_lnb[0]; a.lnb_o = d->d_lnb[1];
  a.M = Mp<T>(d); a.g = d->a3 ? gp<T>(d) : nullptr; a.Bg = d->a3 ? Bgp<T>(d) : nullptr;
  a.Ainv = d->a3 ? Ainvp<T>(d) : nullptr; a.b = b; a.v = v;
  a.work = lwork<T>(d, 0);
  a.acc = d->coop_partial;                                   // [3][COOP_NV] accumulators
  a.err = d->coop_err;
  a.vec_rows = 0;
  DW_CUDA(cudaMemsetAsync(d->coop_partial, 0, 3 * COOP_NV * sizeof(double), s));
  a.out = d->coop_out + (d->defer_slot >= 0 ? 2 * d->defer_slot : 0);
  a.tol = tol;
  void* args[] = {&a};
  cudaError_t le = cudaSuccess;
  size_t dsm = coop_dyn_smem<T>(d->coop_grid);
  if (!d->coop_ring || sizeof(T) == 8) {
    // register-pipelined hops leave shared memory free for the CTA's vector slices
    const int rows = (d->Ne + d->coop_grid - 1) / d->coop_grid;
    const size_t extra = coop_vec_smem<T>(rows, d->Ns, nkv);
    if (dsm + extra <= coop_vec_smem_max<T>()) {
      a.vec_rows = rows;
      dsm += extra;
    }
  }
  if constexpr (sizeof(T) == 8) {
    NS_DISPATCH_FEW(d->Ns, (le = cudaLaunchCooperativeKernel((void*)little_gcr_coop_kernel<T, NSV>, d->coop_grid,
                                                       COOP_THREADS, args, dsm, s)));
  } else {
    bool done = false;
    if (d->coop_ring) {
      NS_DISPATCH_FEW(d->Ns, if constexpr (NSV > 0) {
        le = cudaLaunchCooperativeKernel((void*)little_gcr_coop_kernel<float, NSV, true>, d->coop_grid, COOP_THREADS,
                                         args, coop_ring_smem<NSV>(), s);
        done = true;
      });
    }
    if (!done)
      NS_DISPATCH(d->Ns, (le = cudaLaunchCooperativeKernel((void*)little_gcr_coop_kernel<T, NSV>, d->coop_grid,
                                                         COOP_THREADS, args, dsm, s)));
  }
  DW_CUDA(le);
  dw_note_launch();
  if (d->defer_slot >= 0) {   // results collected later by little_collect
    *iters = 0;
    *relres = 0;
    return DW_OK;
  }
  double h[2];
  int rc = sync_read(d->c, d->coop_out, 2, h, s);
  if (rc) return rc;
  *iters = (int)h[0];
  *relres = h[1];
  return h[1] <= tol ? DW_OK : DW_ENOTCONV;
}

// Solve B^ v_e = b_e, deflated by the global modes (A.3) when available.
// work: 2*nkv + 4 vectors of Ne*Ns complex.
template <typename T>
static int little_gcr(dfl_ctx* d, const T* b, T* v, double tol, int maxit, int nkv, int* iters, double* relres,
                      cudaStream_t s) {
  if (d->coop_grid > 0 && nkv <= COOP_NKV && coop_enabled())
    return little_gcr_coop<T>(d, b, v, tol, maxit, nkv, iters, relres, s);
  const size_t n = (size_t)d->Ne * d->Ns;
  T* work = lwork<T>(d, 0);
  T* tmpo = lwork<T>(d, 2 * nkv + 3);
  T* rhs = lwork<T>(d, 2 * nkv + 4);
  T* t = lwork<T>(d, 2 * nkv + 2);     // the generic GCR's scratch slot, free after it returns
  cudaStream_t st = s;
  int rc;
  DW_CUDA(cudaMemcpyAsync(rhs, b, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s));
  if (d->a3 && (rc = little_PL<T>(d, rhs, s))) return rc;
  auto op = [&](const T* x, T* y) -> int {
    apply_bhat<T>(d, x, tmpo, y, st);
    return d->a3 ? little_PL<T>(d, y, st) : DW_OK;
  };
  int grc = gcr_small<T>(d->c, op, rhs, v, n, work, tol, maxit, nkv, iters, relres, s);
  if (grc < 0) return grc;
  if (d->a3) {
    // v = P~_R chi + g A~^{-1} g^+ b = chi + g A~^{-1} g^+ (b - B^ chi)
    apply_bhat<T>(d, v, tmpo, t, s);
    DW_CUDA(cudaMemcpyAsync(rhs, b, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    blas_axpy<T>(t, rhs, -1.0, 0.0, n, s);
    if ((rc = little_coarse_add<T>(d, rhs, v, s))) return rc;
  }
  return grc;
}

static int ensure_little_work(dfl_ctx* d, int prec, int nkv) {
  size_t count = (size_t)2 * nkv + 10;
  size_t n = (size_t)d->Ne * d->Ns * 2;
  if (d->lw[prec] && d->lw_count >= count) return DW_OK;
  for (int p = 0; p < 2; ++p)
    if (d->lw[p]) { cudaFree(d->lw[p]); d->lw[p] = nullptr; }
  d->lw_count = count;
  DW_CUDA(cudaMalloc(&d->lw[DW_F64], count * n * sizeof(double)));
  DW_CUDA(cudaMalloc(&d->lw[DW_F32], count * n * sizeof(float)));
  return DW_OK;
}

// Appendix A.2 fallback: an ill-conditioned diagonal block -> GCR on the full little system
template <typename T>
static const T* Bp(dfl_ctx* d);
template <> const float* Bp<float>(dfl_ctx* d) { return d->B32; }
template <> const double* Bp<double>(dfl_ctx* d) { return d->B64; }

template <typename T, int NS>
__global__ void little_full_t_kernel(int Nb, int Ns, const int* __restrict__ bnb, const T* __restrict__ B,
                                     const T* __restrict__ v, T* w) {
  const int L = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (L >= Nb) return;
  const int ns = NS ? NS : Ns;
  const cplx<T>* Bc = reinterpret_cast<const cplx<T>*>(B);
  const cplx<T>* vc = reinterpret_cast<const cplx<T>*>(v);
  cplx<T> acc = {T(0), T(0)};
  for (int part = 0; part < 9; ++part) {
    const int src = part == 0 ? L : bnb[L * 8 + part - 1];
    acc = warp_mv<T, NS>(Bc + ((size_t)L * 9 + part) * ns * ns, vc + (size_t)src * ns, ns, lane, acc);
  }
  if (lane < ns) reinterpret_cast<cplx<T>*>(w)[(size_t)L * ns + lane] = acc;
}

template <typename T>
static int little_full_solve(dfl_ctx* d, const T* w, T* v, double tol, int maxit, int nkv, int* iters,
                             double* relres, cudaStream_t s) {
  constexpr int P = prec_of<T>();
  const size_t n = (size_t)d->N;
  if (!d->fw[P]) DW_CUDA(cudaMalloc(&d->fw[P], (size_t)(2 * nkv + 3) * n * 2 * sizeof(T)));
  auto op = [&](const T* x, T* y) -> int {
    NS_DISPATCH(d->Ns, (little_full_t_kernel<T, NSV><<<warps_grid(d->Nb), 128, 0, s>>>(d->Nb, d->Ns, d->d_bnb,
                                                                                      Bp<T>(d), x, y)));
    dw_note_launch();
    return DW_OK;
  };
  return gcr_small<T>(d->c, op, w, v, n, (T*)d->fw[P], tol, maxit, nkv, iters, relres, s);
}

// Full little solve A v = w (prec T; w, v: [Nb][Ns] complex of T)
template <typename T>
static int little_solve_t(dfl_ctx* d, const T* w, T* v, double tol, int maxit, int nkv, int* iters, double* relres,
                          cudaStream_t s) {
  int rc = ensure_little_work(d, prec_of<T>(), nkv);
  if (rc) return rc;
  const int Ns = d->Ns;
  size_t n_e = (size_t)d->Ne * Ns, n_o = (size_t)d->No * Ns;
  if (d->illcond) return little_full_solve<T>(d, w, v, tol, maxit, nkv, iters, relres, s);
  T* we = lwork<T>(d, 2 * nkv + 5);
  T* wo = lwork<T>(d, 2 * nkv + 6);
  T* yo = lwork<T>(d, 2 * nkv + 7);
  T* wt = lwork<T>(d, 2 * nkv + 8);
  unsigned ge = (unsigned)((n_e + 255) / 256), go = (unsigned)((n_o + 255) / 256);
  little_gather_kernel<T, T><<<ge, 256, 0, s>>>(d->Ne, Ns, d->d_list[0], w, we); dw_note_launch();
  little_gather_kernel<T, T><<<go, 256, 0, s>>>(d->No, Ns, d->d_list[1], w, wo); dw_note_launch();
  // yo = B_oo^{-1} w_o ; wt = B_ee^{-1} w_e - M_eo yo
  NS_DISPATCH(Ns, (little_bdiag_kernel<T, NSV><<<warps_grid(d->No), 128, 0, s>>>(d->No, Ns, d->d_list[1],
                                                                             Binvp<T>(d), wo, yo)));
  NS_DISPATCH(Ns, (little_bdiag_kernel<T, NSV><<<warps_grid(d->Ne), 128, 0, s>>>(d->Ne, Ns, d->d_list[0],
                                                                             Binvp<T>(d), we, wt)));
  NS_DISPATCH(Ns, (little_hop_kernel<T, NSV><<<d->Ne, 256, 0, s>>>(d->Ne, Ns, d->d_list[0],
                                                                           d->d_lnb[0], Mp<T>(d), yo, wt, we)));
  dw_note_launch(); dw_note_launch(); dw_note_launch();
  // we now holds w~_e ; solve B^ v_e = w~_e into wt
  rc = little_gcr<T>(d, we, wt, tol, maxit, nkv, iters, relres, s);
  if (rc < 0) return rc;
  // v_o = yo - M_oe v_e  -> into wo
  NS_DISPATCH(Ns, (little_hop_kernel<T, NSV><<<d->No, 256, 0, s>>>(d->No, Ns, d->d_list[1],
                                                                           d->d_lnb[1], Mp<T>(d), wt, yo, wo)));
  dw_note_launch();
  little_scatter_kernel<T, T><<<ge, 256, 0, s>>>(d->Ne, Ns, d->d_list[0], wt, v); dw_note_launch();
  little_scatter_kernel<T, T><<<go, 256, 0, s>>>(d->No, Ns, d->d_list[1], wo, v); dw_note_launch();
  DW_CUDA(cudaGetLastError());
  return rc;
}
int little_solve_f32(dfl_ctx* d, const float* w, float* v, double tol, int maxit, int nkv, int* it, double* rr,
                     cudaStream_t s) {
  return little_solve_t(d, w, v, tol, maxit, nkv, it, rr, s);
}
int little_solve_f64(dfl_ctx* d, const double* w, double* v, double tol, int maxit, int nkv, int* it, double* rr,
                     cudaStream_t s) {
  return little_solve_t(d, w, v, tol, maxit, nkv, it, rr, s);
}
int dfl_nlittle(const dfl_ctx* d) { return d->N; }
dw_ctx* dfl_operator(const dfl_ctx* d) { return d->c; }
// FP64-accurate solution of A v = w (little operator (3.2)/(A.1)) by mixed-precision iterative
// refinement: FP32 even-odd deflated GCR solves for the corrections, FP64 residuals w - A v with the
// FP64 operator.  Used for the restart corrections of the mixed-precision solver, so every little
// GCR iteration runs in FP32 while the correction reaches the outer tolerance.
int little_solve_refined(dfl_ctx* d, const double* w, double* v, double tol, int maxit, int nkv, int* iters,
                         double* relres, cudaStream_t s) {
  const size_t N = d->N;
  if (!d->ref64) DW_CUDA(cudaMalloc(&d->ref64, 3 * N * 2 * sizeof(double)));
  if (!d->ref32) DW_CUDA(cudaMalloc(&d->ref32, 2 * N * 2 * sizeof(float)));
  double* r = d->ref64;
  double* t = r + 2 * N;
  float* w32 = d->ref32;
  float* v32 = w32 + 2 * N;
  double* dres = d->c->d_red + 65536 + 2048;
  double h[3];
  int rc;
  DW_CUDA(cudaMemsetAsync(v, 0, N * 2 * sizeof(double), s));
  DW_CUDA(cudaMemcpyAsync(r, w, N * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  blas_dot<double>(d->c, w, w, N, dres, s);
  if ((rc = sync_read(d->c, dres, 3, h, s))) return rc;
  const double wn = sqrt(h[2]);
  *iters = 0;
  *relres = 0;
  if (wn == 0.0) return DW_OK;
  double rn = wn;
  for (int step = 0; step < 8 && rn > tol * wn && *iters < maxit; ++step) {
    blas_convert<double, float>(r, w32, 1.0 / rn, N, s);
    int it = 0;
    double rr = 0;
    rc = little_solve_t<float>(d, w32, v32, 1e-6, maxit - *iters, nkv, &it, &rr, s);
    if (rc < 0) return rc;
    *iters += it;
    blas_convert<float, double>(v32, t, rn, N, s);
    blas_axpy<double>(t, v, 1.0, 0.0, N, s);
    NS_DISPATCH(d->Ns, (little_full_t_kernel<double, NSV><<<warps_grid(d->Nb), 128, 0, s>>>(
                            d->Nb, d->Ns, d->d_bnb, d->B64, v, t)));
    dw_note_launch();
    DW_CUDA(cudaMemcpyAsync(r, w, N * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    blas_axpy<double>(t, r, -1.0, 0.0, N, s);
    blas_dot<double>(d->c, r, r, N, dres, s);
    if ((rc = sync_read(d->c, dres, 3, h, s))) return rc;
    rn = sqrt(h[2]);
  }
  *relres = rn / wn;
  return rn <= tol * wn ? DW_OK : DW_ENOTCONV;
}

// nrhs FP32 little solves queued back to back; one host synchronisation collects the counts.
// Uses the cooperative solver when available (otherwise each solve synchronises on its own).
template <int NS>
static bool launch_little_mrhs(dfl_ctx* d, CoopMArgs& a, cudaStream_t s, cudaError_t* err) {
  if constexpr (NS == 0) {
    return false;
  } else {
    void* args[] = {&a};
    void* fn = a.RP == 2   ? (void*)little_gcr_coop_mrhs_kernel<NS, 2>
               : a.RP == 4 ? (void*)little_gcr_coop_mrhs_kernel<NS, 4>
               : a.RP == 8 ? (void*)little_gcr_coop_mrhs_kernel<NS, 8>
                           : (void*)little_gcr_coop_mrhs_kernel<NS, 16>;
    *err = cudaLaunchCooperativeKernel(fn, d->coop_grid, COOP_THREADS, args, coop_m_dyn_bytes(NS, a.RP), s);
    return true;
  }
}

// shared-memory limits of the multi-RHS kernels (RP = 2, 4, 8, 16); CTAs per SM of the largest
template <int NS>
static int mrhs_prepare(size_t dsm_max) {
  if constexpr (NS == 0) {
    return 0;
  } else {
    const void* fns[4] = {(const void*)little_gcr_coop_mrhs_kernel<NS, 2>, (const void*)little_gcr_coop_mrhs_kernel<NS, 4>,
                          (const void*)little_gcr_coop_mrhs_kernel<NS, 8>, (const void*)little_gcr_coop_mrhs_kernel<NS, 16>};
    for (int q = 0; q < 4; ++q)
      if (cudaFuncSetAttribute(fns[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coop_m_dyn_bytes(NS, 2 << q)) !=
          cudaSuccess)
        return 0;
    int bm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, fns[3], COOP_THREADS, dsm_max) != cudaSuccess) return 0;
    return bm;
  }
}

// The R (<= COOP_MAXR) even-odd reduced little systems of a batch in one multi-RHS cooperative
// launch: the per-RHS even-odd preparation and reconstruction (A.2) around it as in little_solve_t.
static int little_solve_mrhs(dfl_ctx* d, const float* w, float* v, const double* tol, const int* idx, int R,
                             int maxit, int nkv, int* iters, double* relres, cudaStream_t s) {
  const int Ns = d->Ns;
  const size_t n_e = (size_t)d->Ne * Ns, n_o = (size_t)d->No * Ns, N2 = (size_t)d->N * 2;
  float* bE = d->mio;                                   // [R][n_e] complex right-hand sides
  float* vE = d->mio + (size_t)COOP_MAXR * n_e * 2;     // [R][n_e] complex solutions
  float* wO = d->meo;                                   // [R][n_o] complex
  float* yO = d->meo + (size_t)COOP_MAXR * n_o * 2;
  unsigned ge = (unsigned)((n_e + 255) / 256), go = (unsigned)((n_o + 255) / 256);
  // systems idx[0], idx[0] + 1, ...: every step below is one launch for all of them (grid.y)
  bool contiguous = true;
  for (int q = 1; q < R; ++q) contiguous &= idx[q] == idx[0] + q;
  if (contiguous) {
    const float* wr = w + (size_t)idx[0] * N2;
    const size_t se = 2 * (size_t)n_e, so = 2 * (size_t)n_o;
    float* wt = vE;                                     // scratch until the solve overwrites it
    little_gather_kernel<float, float><<<dim3(ge, R), 256, 0, s>>>(d->Ne, Ns, d->d_list[0], wr, bE, N2, se);
    little_gather_kernel<float, float><<<dim3(go, R), 256, 0, s>>>(d->No, Ns, d->d_list[1], wr, wO, N2, so);
    NS_DISPATCH(Ns, (little_bdiag_kernel<float, NSV><<<dim3(warps_grid(d->No), R), 128, 0, s>>>(
                         d->No, Ns, d->d_list[1], d->Binv32, wO, yO, so)));
    NS_DISPATCH(Ns, (little_bdiag_kernel<float, NSV><<<dim3(warps_grid(d->Ne), R), 128, 0, s>>>(
                         d->Ne, Ns, d->d_list[0], d->Binv32, bE, wt, se)));
    NS_DISPATCH(Ns, (little_hop_kernel<float, NSV><<<dim3(d->Ne, R), 256, 0, s>>>(
                         d->Ne, Ns, d->d_list[0], d->d_lnb[0], d->M32, yO, wt, bE, so, se)));
    for (int q = 0; q < 5; ++q) dw_note_launch();
  }
  for (int q = 0; q < R && !contiguous; ++q) {
    const float* wr = w + (size_t)idx[q] * N2;
    float* be = bE + (size_t)q * n_e * 2;
    float* wo = wO + (size_t)q * n_o * 2;
    float* yo = yO + (size_t)q * n_o * 2;
    float* wt = vE + (size_t)q * n_e * 2;               // scratch until the solve overwrites it
    little_gather_kernel<float, float><<<ge, 256, 0, s>>>(d->Ne, Ns, d->d_list[0], wr, be); dw_note_launch();
    little_gather_kernel<float, float><<<go, 256, 0, s>>>(d->No, Ns, d->d_list[1], wr, wo); dw_note_launch();
    NS_DISPATCH(Ns, (little_bdiag_kernel<float, NSV><<<warps_grid(d->No), 128, 0, s>>>(d->No, Ns, d->d_list[1],
                                                                                d->Binv32, wo, yo)));
    NS_DISPATCH(Ns, (little_bdiag_kernel<float, NSV><<<warps_grid(d->Ne), 128, 0, s>>>(d->Ne, Ns, d->d_list[0],
                                                                                d->Binv32, be, wt)));
    NS_DISPATCH(Ns, (little_hop_kernel<float, NSV><<<d->Ne, 256, 0, s>>>(d->Ne, Ns, d->d_list[0], d->d_lnb[0],
                                                                         d->M32, yo, wt, be)));
    dw_note_launch(); dw_note_launch(); dw_note_launch();
  }
  float htol[COOP_MAXR];
  for (int q = 0; q < R; ++q) htol[q] = (float)tol[idx[q]];
  DW_CUDA(cudaMemcpyAsync(d->mtol, htol, R * sizeof(float), cudaMemcpyHostToDevice, s));
  CoopMArgs a;
  a.Ne = d->Ne; a.No = d->No; a.nkv = nkv; a.maxit = maxit; a.a3 = d->a3 ? 1 : 0; a.R = R; a.RP = coop_mrp(R);
  a.list_e = d->d_list[0]; a.list_o = d->d_list[1]; a.lnb_e = d->d_lnb[0]; a.lnb_o = d->d_lnb[1];
  a.M = d->M32; a.g = d->a3 ? d->g32 : nullptr; a.Bg = d->a3 ? d->Bg32 : nullptr; a.Ainv = d->a3 ? d->Ainv32 : nullptr;
  a.b = bE; a.tol = d->mtol; a.v = vE; a.work = d->mw; a.scratch = d->mscr; a.acc = d->macc; a.out = d->mout;
  DW_CUDA(cudaMemsetAsync(d->macc, 0, 3 * COOP_MNV * sizeof(double), s));
  cudaError_t le = cudaSuccess;
  bool launched = false;
  NS_DISPATCH_FEW(Ns, (launched = launch_little_mrhs<NSV>(d, a, s, &le)));
  if (!launched) { dw_set_error("multi-RHS little solver: unsupported Ns"); return DW_EINVAL; }
  DW_CUDA(le);
  dw_note_launch();
  if (contiguous) {
    float* vr = v + (size_t)idx[0] * N2;
    const size_t se = 2 * (size_t)n_e, so = 2 * (size_t)n_o;
    NS_DISPATCH(Ns, (little_hop_kernel<float, NSV><<<dim3(d->No, R), 256, 0, s>>>(
                         d->No, Ns, d->d_list[1], d->d_lnb[1], d->M32, vE, yO, wO, se, so)));
    little_scatter_kernel<float, float><<<dim3(ge, R), 256, 0, s>>>(d->Ne, Ns, d->d_list[0], vE, vr, se, N2);
    little_scatter_kernel<float, float><<<dim3(go, R), 256, 0, s>>>(d->No, Ns, d->d_list[1], wO, vr, so, N2);
    for (int q = 0; q < 3; ++q) dw_note_launch();
  }
  for (int q = 0; q < R && !contiguous; ++q) {
    float* vr = v + (size_t)idx[q] * N2;
    float* ve = vE + (size_t)q * n_e * 2;
    float* wo = wO + (size_t)q * n_o * 2;
    float* yo = yO + (size_t)q * n_o * 2;
    NS_DISPATCH(Ns, (little_hop_kernel<float, NSV><<<d->No, 256, 0, s>>>(d->No, Ns, d->d_list[1], d->d_lnb[1],
                                                                         d->M32, ve, yo, wo)));
    dw_note_launch();
    little_scatter_kernel<float, float><<<ge, 256, 0, s>>>(d->Ne, Ns, d->d_list[0], ve, vr); dw_note_launch();
    little_scatter_kernel<float, float><<<go, 256, 0, s>>>(d->No, Ns, d->d_list[1], wo, vr); dw_note_launch();
  }
  double h[2 * COOP_MAXR];
  int rc = sync_read(d->c, d->mout, 2 * R, h, s);
  if (rc) return rc;
  for (int q = 0; q < R; ++q) {
    iters[idx[q]] = (int)h[2 * q];
    relres[idx[q]] = h[2 * q + 1];
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

static bool mrhs_enabled() {
  const char* e = getenv("DW_LITTLE_MRHS");
  return !(e && e[0] == '0');
}

int little_solve_batch_f32(dfl_ctx* d, const float* w, float* v, const double* tol, const int* use, int maxit,
                           int nkv, int nrhs, int* iters, double* relres, cudaStream_t s) {
  const size_t N2 = (size_t)d->N * 2;
  for (int r = 0; r < nrhs; ++r) { iters[r] = 0; relres[r] = 0; }
  if (d->coop_m && !d->illcond && nkv <= COOP_NKV && coop_enabled() && mrhs_enabled()) {
    std::vector<int> idx;
    for (int r = 0; r < nrhs; ++r)
      if (use[r]) idx.push_back(r);
    for (size_t q0 = 0; q0 < idx.size(); q0 += COOP_MAXR) {
      const int R = (int)std::min<size_t>(COOP_MAXR, idx.size() - q0);
      int rc = little_solve_mrhs(d, w, v, tol, idx.data() + q0, R, maxit, nkv, iters, relres, s);
      if (rc < 0) return rc;
    }
    return DW_OK;
  }
  const bool coop = d->coop_grid > 0 && nkv <= COOP_NKV && coop_enabled() && !d->illcond && nrhs <= 64;
  for (int r = 0; r < nrhs; ++r) {
    if (!use[r]) continue;
    d->defer_slot = coop ? r : -1;
    int rc = little_solve_t<float>(d, w + r * N2, v + r * N2, tol[r], maxit, nkv, iters + r, relres + r, s);
    d->defer_slot = -1;
    if (rc < 0) return rc;
  }
  if (coop) {
    std::vector<double> h(2 * nrhs);
    int rc = sync_read(d->c, d->coop_out, 2 * nrhs, h.data(), s);
    if (rc) return rc;
    for (int r = 0; r < nrhs; ++r)
      if (use[r]) { iters[r] = (int)h[2 * r]; relres[r] = h[2 * r + 1]; }
  }
  return DW_OK;
}


// little_solve_refined for nrhs systems at once: FP64 residuals per right-hand side, the FP32
// correction solves of every refinement step batched (multi-RHS cooperative solver).
int little_solve_refined_batch(dfl_ctx* d, const double* w, double* v, double tol, const int* use, int maxit,
                               int nkv, int nrhs, int* iters, double* relres, cudaStream_t s) {
  const size_t N = d->N, N2 = N * 2;
  double* r64 = nullptr;
  double* t64 = nullptr;
  float* w32 = nullptr;
  float* v32 = nullptr;
  DW_CUDA(cudaMallocAsync(&r64, nrhs * N2 * sizeof(double), s));
  DW_CUDA(cudaMallocAsync(&t64, nrhs * N2 * sizeof(double), s));
  DW_CUDA(cudaMallocAsync(&w32, nrhs * N2 * sizeof(float), s));
  DW_CUDA(cudaMallocAsync(&v32, nrhs * N2 * sizeof(float), s));
  double* dres = d->c->d_red + 65536 + 2048;
  std::vector<double> h(3 * nrhs), wn(nrhs, 0.0), rn(nrhs, 0.0), t32(nrhs, 1e-6);
  std::vector<int> act(nrhs, 0), it(nrhs, 0);
  std::vector<double> rr(nrhs, 0.0);
  int rc = DW_OK;
  auto norms = [&](const double* x) -> int {
    for (int r = 0; r < nrhs; ++r) blas_dot<double>(d->c, x + r * N2, x + r * N2, N, dres + 3 * r, s);
    return sync_read(d->c, dres, 3 * nrhs, h.data(), s);
  };
  for (int r = 0; r < nrhs; ++r) {
    iters[r] = 0;
    relres[r] = 0.0;
    DW_CUDA(cudaMemsetAsync(v + r * N2, 0, N2 * sizeof(double), s));
  }
  DW_CUDA(cudaMemcpyAsync(r64, w, nrhs * N2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if ((rc = norms(w))) goto done;
  for (int r = 0; r < nrhs; ++r) { wn[r] = sqrt(h[3 * r + 2]); rn[r] = wn[r]; }
  for (int step = 0; step < 8; ++step) {
    int any = 0;
    for (int r = 0; r < nrhs; ++r) {
      act[r] = use[r] && wn[r] > 0.0 && rn[r] > tol * wn[r] && iters[r] < maxit;
      any |= act[r];
      if (act[r]) blas_convert<double, float>(r64 + r * N2, w32 + r * N2, 1.0 / rn[r], N, s);
    }
    if (!any) break;
    int mx = maxit;
    for (int r = 0; r < nrhs; ++r)
      if (act[r]) mx = std::min(mx, maxit - iters[r]);
    if ((rc = little_solve_batch_f32(d, w32, v32, t32.data(), act.data(), std::max(mx, 1), nkv, nrhs, it.data(),
                                     rr.data(), s)) < 0)
      goto done;
    rc = DW_OK;
    for (int r = 0; r < nrhs; ++r) {
      if (!act[r]) continue;
      iters[r] += it[r];
      blas_convert<float, double>(v32 + r * N2, t64 + r * N2, rn[r], N, s);
      blas_axpy<double>(t64 + r * N2, v + r * N2, 1.0, 0.0, N, s);
      NS_DISPATCH(d->Ns, (little_full_t_kernel<double, NSV><<<warps_grid(d->Nb), 128, 0, s>>>(
                              d->Nb, d->Ns, d->d_bnb, d->B64, v + r * N2, t64 + r * N2)));
      dw_note_launch();
      DW_CUDA(cudaMemcpyAsync(r64 + r * N2, w + r * N2, N2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      blas_axpy<double>(t64 + r * N2, r64 + r * N2, -1.0, 0.0, N, s);
    }
    if ((rc = norms(r64))) goto done;
    for (int r = 0; r < nrhs; ++r)
      if (act[r]) rn[r] = sqrt(h[3 * r + 2]);
  }
  for (int r = 0; r < nrhs; ++r) {
    relres[r] = wn[r] > 0.0 ? rn[r] / wn[r] : 0.0;
    if (use[r] && rn[r] > tol * wn[r]) rc = DW_ENOTCONV;
  }
done:
  cudaFreeAsync(r64, s);
  cudaFreeAsync(t64, s);
  cudaFreeAsync(w32, s);
  cudaFreeAsync(v32, s);
  return rc;
}

extern "C" int little_dirac_solve(dfl_ctx* d, int prec, const void* w, void* v, double tol, int maxit, int* iters,
                                  double* relres, void* stream) {
  if (!d || !w || !v || w == v || (prec != DW_F32 && prec != DW_F64) || maxit < 1 || !(tol > 0)) {
    dw_set_error("little_dirac_solve: bad argument");
    return DW_EINVAL;
  }
  int it = 0;
  double rr = 0;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prec == DW_F64 ? little_solve_t(d, (const double*)w, (double*)v, tol, maxit, 24, &it, &rr, s)
                          : little_solve_t(d, (const float*)w, (float*)v, tol, maxit, 24, &it, &rr, s);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  if (rc >= 0) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dw_cuda_fail(e, "little_dirac_solve");
  }
  return rc;
}

// Shape sweep of the FP32 cooperative little solver: grid sizes (all SMs, 3/4 and 1/2 of them, each
// CTA then owning more block rows) x hop variant (shared-memory ring / register pipeline), timed
// with CUDA events on little solves of a fixed random right-hand side to 1e-6; the fastest per
// iteration is kept in the context.
extern "C" int dfl_autotune(dfl_ctx* d, char* report, size_t report_len) {
  if (!d) { dw_set_error("dfl_autotune: null context"); return DW_EINVAL; }
  if (int rc = dw_check_device(d->c, "dfl_autotune")) return rc;
  if (d->coop_grid <= 0 || d->illcond) {
    if (report && report_len) snprintf(report, report_len, "{\"tuned\": false}");
    return DW_OK;
  }
  cudaStream_t s = 0;
  const size_t n2 = (size_t)d->N * 2;
  float *w = nullptr, *v = nullptr;
  DW_CUDA(cudaMalloc(&w, n2 * sizeof(float)));
  DW_CUDA(cudaMalloc(&v, n2 * sizeof(float)));
  {
    std::vector<float> hw(n2);
    uint64_t x = 0x9e3779b97f4a7c15ull;
    for (auto& e : hw) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; e = (float)((double)(x >> 11) / 9007199254740992.0 - 0.5); }
    DW_CUDA(cudaMemcpy(w, hw.data(), n2 * sizeof(float), cudaMemcpyHostToDevice));
  }
  const int full = d->coop_grid;
  const bool ring_ok = d->coop_ring;
  int best_grid = full;
  bool best_ring = ring_ok;
  double best = 1e300;
  std::string rep = "{\"tuned\": true, \"us_per_iteration\": {";
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  bool first = true;
  for (int gi = 0; gi < 3; ++gi) {
    const int grid = gi == 0 ? full : (gi == 1 ? full * 3 / 4 : full / 2);
    for (int rv = (ring_ok ? 1 : 0); rv >= 0; --rv) {
      d->coop_grid = grid;
      d->coop_ring = rv == 1;
      int it = 0;
      double rr = 0;
      int rc = little_solve_t<float>(d, w, v, 1e-6, 2000, 24, &it, &rr, s);   // warm-up
      if (rc < 0) { cudaFree(w); cudaFree(v); d->coop_grid = full; d->coop_ring = ring_ok; return rc; }
      cudaEventRecord(e0, s);
      int tot = 0;
      for (int r = 0; r < 3; ++r) {
        little_solve_t<float>(d, w, v, 1e-6, 2000, 24, &it, &rr, s);
        tot += it;
      }
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1e3 * ms / std::max(tot, 1);
      char buf[96];
      snprintf(buf, sizeof buf, "%s\"grid %d %s\": %.2f", first ? "" : ", ", grid, rv ? "ring" : "registers", us);
      rep += buf;
      first = false;
      if (us < best) { best = us; best_grid = grid; best_ring = rv == 1; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(w);
  cudaFree(v);
  d->coop_grid = best_grid;
  d->coop_ring = best_ring;
  char tail[128];
  snprintf(tail, sizeof tail, "}, \"grid\": %d, \"ring\": %d}", best_grid, best_ring ? 1 : 0);
  rep += tail;
  if (report && report_len) snprintf(report, report_len, "%s", rep.c_str());
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

extern "C" int little_dirac_solve_batch(dfl_ctx* d, int prec, int nrhs, const void* w, void* v, double tol,
                                        int maxit, int* iters, double* relres, void* stream) {
  if (!d || !w || !v || w == v || nrhs < 1 || nrhs > 64 || (prec != DW_F32 && prec != DW_F64) || maxit < 1 ||
      !(tol > 0)) {
    dw_set_error("little_dirac_solve_batch: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> use(nrhs, 1), it(nrhs, 0);
  std::vector<double> rr(nrhs, 0.0), tl(nrhs, tol);
  int rc = prec == DW_F32
               ? little_solve_batch_f32(d, (const float*)w, (float*)v, tl.data(), use.data(), maxit, 24, nrhs,
                                        it.data(), rr.data(), s)
               : little_solve_refined_batch(d, (const double*)w, (double*)v, tol, use.data(), maxit, 24, nrhs,
                                            it.data(), rr.data(), s);
  if (rc < 0) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return dw_cuda_fail(e, "little_dirac_solve_batch");
  for (int r = 0; r < nrhs; ++r) {
    if (iters) iters[r] = it[r];
    if (relres) relres[r] = rr[r];
    if (prec == DW_F32 && !(rr[r] <= tol)) rc = DW_ENOTCONV;
  }
  return rc;
}

// ---------------------------------------------------------------------- build
// Block tables of the deflation blocks (neighbours, Schwarz blocks of each block, parity lists
// and neighbour positions) on the device; the host keeps the even-block list.
static int build_tables(dw_ctx* c, dfl_ctx* d) {
  const Geom& g = c->g;
  // ---- tables
  std::vector<int> bcoord((size_t)d->Nb * 4), sap2dfl(g.nsap), sub((size_t)d->Nb * d->nsub, -1), fill(d->Nb, 0),
      bnb((size_t)d->Nb * 8);
  for (int L = 0; L < d->Nb; ++L) {
    int r = L;
    for (int mu = 3; mu >= 0; --mu) { bcoord[L * 4 + mu] = r % d->nb[mu]; r /= d->nb[mu]; }
    for (int dd = 0; dd < 8; ++dd) {
      int mu = dd / 2, sg = (dd & 1) ? -1 : 1;
      int nc[4] = {bcoord[L * 4], bcoord[L * 4 + 1], bcoord[L * 4 + 2], bcoord[L * 4 + 3]};
      nc[mu] = (nc[mu] + sg + d->nb[mu]) % d->nb[mu];
      bnb[L * 8 + dd] = ((nc[0] * d->nb[1] + nc[1]) * d->nb[2] + nc[2]) * d->nb[3] + nc[3];
    }
  }
  for (int b = 0; b < g.nsap; ++b) {
    int r = b, bc[4];
    for (int mu = 3; mu >= 0; --mu) { bc[mu] = r % c->nsb[mu]; r /= c->nsb[mu]; }
    int dc[4];
    for (int mu = 0; mu < 4; ++mu) dc[mu] = bc[mu] * g.sb[mu] / d->bs[mu];
    int L = ((dc[0] * d->nb[1] + dc[1]) * d->nb[2] + dc[2]) * d->nb[3] + dc[3];
    sap2dfl[b] = L;
    sub[(size_t)L * d->nsub + fill[L]++] = b;
  }
  // parity lists and neighbour positions
  std::vector<int> list[2], pos(d->Nb);
  for (int L = 0; L < d->Nb; ++L) {
    int par = (bcoord[L * 4] + bcoord[L * 4 + 1] + bcoord[L * 4 + 2] + bcoord[L * 4 + 3]) & 1;
    pos[L] = (int)list[par].size();
    list[par].push_back(L);
  }
  d->Ne = (int)list[0].size();
  d->No = (int)list[1].size();
  std::vector<int> lnb[2];
  for (int par = 0; par < 2; ++par)
    for (int L : list[par])
      for (int dd = 0; dd < 8; ++dd) lnb[par].push_back(pos[bnb[L * 8 + dd]]);
  auto up = [&](int** dst, const std::vector<int>& v) -> int {
    DW_CUDA(cudaMalloc(dst, v.size() * sizeof(int)));
    DW_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
    return DW_OK;
  };
  int rc;
  if ((rc = up(&d->d_sub, sub)) || (rc = up(&d->d_sap2dfl, sap2dfl)) || (rc = up(&d->d_bnb, bnb)) ||
      (rc = up(&d->d_list[0], list[0])) || (rc = up(&d->d_list[1], list[1])) || (rc = up(&d->d_lnb[0], lnb[0])) ||
      (rc = up(&d->d_lnb[1], lnb[1])))
    return rc;

  d->hlist0 = list[0];
  return DW_OK;
}

// Little Dirac operator (A.1) of the operator of c on the basis held in d (basis64, and basis16 when
// stored in BF16): assembly in FP64 (or the given host copy B64_given), diagonal-block inverses with
// the condition check (A.2), B_LL^{-1} B_LL' products, global-mode deflation (A.3) from the
// restriction coefficients d->graw, and the set-up of the cooperative little solvers.
static int little_setup(dw_ctx* c, dfl_ctx* d, const double* B64_given) {
  const Geom& g = c->g;
  const int Ns = d->Ns;
  const dfl_params* p = &d->p;
  cudaStream_t s = 0;
  int rc;
  // ---- little operator (A.1) from the stored basis, FP64
  const size_t mat = (size_t)Ns * Ns * 2;
  DW_CUDA(cudaMalloc(&d->B64, d->Nb * 9 * mat * sizeof(double)));
  if (B64_given) {
    DW_CUDA(cudaMemcpy(d->B64, B64_given, d->Nb * 9 * mat * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    assemble_kernel<<<(unsigned)(d->Nb * 9 * Ns), 128, 0, s>>>(g, d->d_sub, d->nsub, d->d_sap2dfl, Ns,
                                                              (const double*)c->links[DW_F64],
                                                              (const double*)c->clov[DW_F64], d->basis64, d->B64); dw_note_launch();
  }
  DW_CUDA(cudaGetLastError());
  DW_CUDA(cudaMalloc(&d->B32, d->Nb * 9 * mat * sizeof(float)));
  blas_convert<double, float>(d->B64, d->B32, 1.0, (size_t)d->Nb * 9 * Ns * Ns, s);
  DW_CUDA(cudaMalloc(&d->Binv64, d->Nb * mat * sizeof(double)));
  DW_CUDA(cudaMalloc(&d->Binv32, d->Nb * mat * sizeof(float)));
  DW_CUDA(cudaMalloc(&d->M64, d->Nb * 8 * mat * sizeof(double)));
  DW_CUDA(cudaMalloc(&d->M32, d->Nb * 8 * mat * sizeof(float)));
  double* d_cond;
  DW_CUDA(cudaMalloc(&d_cond, d->Nb * sizeof(double)));
  block_inverse_kernel<<<d->Nb, 32, 0, s>>>(Ns, d->B64, d->Binv64, d->Binv32, d_cond); dw_note_launch();
  size_t tot = (size_t)d->Nb * 8 * Ns * Ns;
  neighbour_products_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d->Nb, Ns, d->B64, d->Binv64, d->M64,
                                                                          d->M32); dw_note_launch();
  std::vector<double> cond(d->Nb);
  DW_CUDA(cudaMemcpyAsync(cond.data(), d_cond, d->Nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  cudaFree(d_cond);
  d->max_cond = 0;
  for (double x : cond) d->max_cond = std::max(d->max_cond, std::isfinite(x) ? x : INFINITY);
  d->illcond = !(d->max_cond <= p->cond_max);

  // ---- global-mode deflation (A.3): g_l = even-block part of Phi^+ psi_l, orthonormalised
  d->a3 = false;
  if (!d->illcond && d->graw.size() == (size_t)Ns * d->Ne * Ns) {
    const size_t ne = (size_t)d->Ne * Ns;
    std::vector<cd> G = d->graw;
    // modified Gram-Schmidt with re-orthogonalisation (host, FP64)
    bool ok = true;
    for (int l = 0; l < Ns && ok; ++l) {
      cd* v = &G[(size_t)l * ne];
      double n0 = 0;
      for (size_t i = 0; i < ne; ++i) n0 += std::norm(v[i]);
      for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < l; ++j) {
          const cd* u = &G[(size_t)j * ne];
          cd z = 0;
          for (size_t i = 0; i < ne; ++i) z += std::conj(u[i]) * v[i];
          for (size_t i = 0; i < ne; ++i) v[i] -= z * u[i];
        }
      double n1 = 0;
      for (size_t i = 0; i < ne; ++i) n1 += std::norm(v[i]);
      if (!(n1 > 1e-24 * n0)) { ok = false; break; }
      double sc = 1.0 / sqrt(n1);
      for (size_t i = 0; i < ne; ++i) v[i] *= sc;
    }
    if (ok) {
      if ((rc = ensure_little_work(d, DW_F64, 24))) return rc;
      DW_CUDA(cudaMalloc(&d->g64, Ns * ne * 2 * sizeof(double)));
      DW_CUDA(cudaMalloc(&d->g32, Ns * ne * 2 * sizeof(float)));
      DW_CUDA(cudaMalloc(&d->Bg64, Ns * ne * 2 * sizeof(double)));
      DW_CUDA(cudaMalloc(&d->Bg32, Ns * ne * 2 * sizeof(float)));
      DW_CUDA(cudaMemcpy(d->g64, G.data(), Ns * ne * sizeof(cd), cudaMemcpyHostToDevice));
      blas_convert<double, float>(d->g64, d->g32, 1.0, Ns * ne, s);
      double* tmpo = lwork<double>(d, 0);
      for (int l = 0; l < Ns; ++l)
        apply_bhat<double>(d, d->g64 + (size_t)l * ne * 2, tmpo, d->Bg64 + (size_t)l * ne * 2, s);
      blas_convert<double, float>(d->Bg64, d->Bg32, 1.0, Ns * ne, s);
      // A~ = g^+ B^ g
      std::vector<cd> Bg((size_t)Ns * ne);
      DW_CUDA(cudaMemcpyAsync(Bg.data(), d->Bg64, Ns * ne * sizeof(cd), cudaMemcpyDeviceToHost, s));
      DW_CUDA(cudaStreamSynchronize(s));
      std::vector<cd> At((size_t)Ns * Ns), X((size_t)Ns * Ns);
      for (int a = 0; a < Ns; ++a)
        for (int b = 0; b < Ns; ++b) {
          cd z = 0;
          for (size_t i = 0; i < ne; ++i) z += std::conj(G[(size_t)a * ne + i]) * Bg[(size_t)b * ne + i];
          At[a * Ns + b] = z;
          X[a * Ns + b] = a == b ? 1.0 : 0.0;
        }
      for (int col = 0; col < Ns && ok; ++col) {   // Gauss-Jordan with partial pivoting
        int piv = col;
        for (int r = col + 1; r < Ns; ++r)
          if (std::abs(At[r * Ns + col]) > std::abs(At[piv * Ns + col])) piv = r;
        if (std::abs(At[piv * Ns + col]) == 0.0) { ok = false; break; }
        for (int b = 0; b < Ns; ++b) { std::swap(At[col * Ns + b], At[piv * Ns + b]); std::swap(X[col * Ns + b], X[piv * Ns + b]); }
        cd pinv = 1.0 / At[col * Ns + col];
        for (int b = 0; b < Ns; ++b) { At[col * Ns + b] *= pinv; X[col * Ns + b] *= pinv; }
        for (int r = 0; r < Ns; ++r) {
          if (r == col) continue;
          cd f = At[r * Ns + col];
          for (int b = 0; b < Ns; ++b) { At[r * Ns + b] -= f * At[col * Ns + b]; X[r * Ns + b] -= f * X[col * Ns + b]; }
        }
      }
      if (ok) {
        d->Atil_inv = X;
        d->a3 = true;
        DW_CUDA(cudaMalloc(&d->Ainv64, (size_t)Ns * Ns * sizeof(cd)));
        DW_CUDA(cudaMalloc(&d->Ainv32, (size_t)Ns * Ns * 2 * sizeof(float)));
        DW_CUDA(cudaMemcpy(d->Ainv64, X.data(), (size_t)Ns * Ns * sizeof(cd), cudaMemcpyHostToDevice));
        blas_convert<double, float>(d->Ainv64, d->Ainv32, 1.0, (size_t)Ns * Ns, s);
      }
    }
  }
  // cooperative little solver: one CTA per SM when all of them can be resident
  {
    int dev = 0, sms = 0, coop = 0, b32 = 0, b64 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const size_t dsm32 = coop_dyn_smem<float>(sms), dsm64 = coop_dyn_smem<double>(sms);
    NS_DISPATCH(Ns, (cudaFuncSetAttribute(little_gcr_coop_kernel<float, NSV>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)coop_vec_smem_max<float>())));
    NS_DISPATCH_FEW(Ns, (cudaFuncSetAttribute(little_gcr_coop_kernel<double, NSV>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)coop_vec_smem_max<double>())));
    NS_DISPATCH(Ns, (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, little_gcr_coop_kernel<float, NSV>,
                                                                   COOP_THREADS, dsm32)));
    NS_DISPATCH_FEW(Ns, (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, little_gcr_coop_kernel<double, NSV>,
                                                                   COOP_THREADS, dsm64)));
    d->coop_grid = (coop && b32 > 0 && b64 > 0 && Ns <= 32) ? sms : 0;
    if (d->coop_grid) {
      DW_CUDA(cudaMalloc(&d->coop_partial, (size_t)2 * coop_gpad(d->coop_grid) * COOP_NV * sizeof(double)));
      DW_CUDA(cudaMalloc(&d->coop_out, 2 * 64 * sizeof(double)));
      DW_CUDA(cudaMalloc(&d->coop_err, sizeof(int)));
      DW_CUDA(cudaMemset(d->coop_err, 0, sizeof(int)));
      // FP32 solver variant with the operator staged through a shared-memory ring (Ns = 8, 20);
      // DW_COOP_RING=0 keeps the register-pipelined hops
      int br = 0;
      NS_DISPATCH_FEW(Ns, if constexpr (NSV > 0) {
        if (cudaFuncSetAttribute(little_gcr_coop_kernel<float, NSV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)coop_ring_smem<NSV>()) == cudaSuccess)
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&br, little_gcr_coop_kernel<float, NSV, true>, COOP_THREADS,
                                                        coop_ring_smem<NSV>());
      });
      cudaGetLastError();
      const char* re = getenv("DW_COOP_RING");
      d->coop_ring = br > 0 && !(re && re[0] == '0');
      // multi-RHS solver (batches of right-hand sides): Ns with a compiled kernel, all CTAs resident
      int bm = 0;
      const size_t dsmm = coop_m_dyn_bytes(Ns, COOP_MRP);
      NS_DISPATCH_FEW(Ns, (bm = mrhs_prepare<NSV>(dsmm)));
      cudaGetLastError();
      if (bm > 0) {
        const size_t ne = (size_t)d->Ne * Ns, no = (size_t)d->No * Ns;
        DW_CUDA(cudaMalloc(&d->mw, ((size_t)2 * COOP_NKV + 6) * COOP_MRP * std::max(ne, no) * 2 * sizeof(float)));
        DW_CUDA(cudaMalloc(&d->mio, (size_t)2 * COOP_MAXR * ne * 2 * sizeof(float)));
        DW_CUDA(cudaMalloc(&d->meo, (size_t)2 * COOP_MAXR * no * 2 * sizeof(float)));
        DW_CUDA(cudaMalloc(&d->macc, (size_t)3 * COOP_MNV * sizeof(double)));
        DW_CUDA(cudaMalloc(&d->mscr, (size_t)sms * coop_m_cta_scratch(Ns) * sizeof(float)));
        DW_CUDA(cudaMalloc(&d->mtol, COOP_MAXR * sizeof(float)));
        DW_CUDA(cudaMalloc(&d->mout, 2 * COOP_MAXR * sizeof(double)));
        d->coop_m = true;
      }
    }
    if ((rc = ensure_little_work(d, DW_F64, COOP_NKV))) return rc;
  }
  return DW_OK;
}

// The bootstrapped steps of the subspace generation (Section 5.3): the Ns fields (packed, precision ip,
// in `work`) are replaced boot_steps times by approximate solutions of D chi_l = psi_l, normalised; each
// approximate solve is the mixed-precision DFL+SAP+GCR solver deflated by the block subspace of the
// current fields (built without further inverse iteration), stopped at ||psi_l - D chi_l|| <=
// boot_tol ||psi_l|| or after boot_nmx GCR steps, the Ns fields in one batch.
static int bootstrap_steps(dw_ctx* c, const dfl_params* p, void* work, int ip, int* steps_done, int* gcr_total) {
  const size_t V = c->V, n = V * 12, fs = V * 24;
  const int Ns = p->Ns;
  cudaStream_t s = 0;
  double *canon = nullptr, *sol = nullptr;
  DW_CUDA(cudaMalloc(&canon, (size_t)Ns * fs * sizeof(double)));
  DW_CUDA(cudaMalloc(&sol, (size_t)Ns * fs * sizeof(double)));
  struct Free { void* a; void* b; ~Free() { cudaFree(a); cudaFree(b); } } guard{canon, sol};
  dfl_params q = *p;
  q.n_inv = 0;
  q.boot_steps = 0;
  q.net_weights = nullptr;
  q.basis_prec = DW_BF16;
  sol_params sp{};
  sp.tol = p->boot_tol;
  sp.nkv = 16;
  sp.nmx = p->boot_nmx > 0 ? p->boot_nmx : 1000;
  sp.ncy = p->ncy;
  sp.nmr = p->nmr;
  sp.mixed = 1;
  sp.inner_rtol = 1e-5;
  sp.little_tol_out = 1e-12;
  sp.little_tol_in = 1e-6;
  sp.little_tol_cap = 1e-1;
  sp.little_nkv = 24;
  sp.little_maxit = 2000;
  std::vector<sol_info> inf(Ns);
  double* dres = c->d_red + 65536 + 20480;
  int rc;
  for (int step = 0; step < p->boot_steps; ++step) {
    if ((rc = dw_unpack(c, ip, Ns, work, canon, s))) return rc;
    dfl_ctx* dt = nullptr;
    rc = deflation_build(c, &q, canon, &dt, nullptr);
    if (rc < 0) return rc;
    rc = gcr_solve(c, dt, &sp, Ns, canon, sol, inf.data(), s);
    dfl_destroy(dt);
    if (rc < 0) return rc;
    for (int l = 0; l < Ns; ++l) {
      *gcr_total += inf[l].iterations;
      blas_dot<double>(c, sol + (size_t)l * fs, sol + (size_t)l * fs, n, dres + 3 * l, s);
    }
    std::vector<double> h(3 * Ns);
    if ((rc = sync_read(c, dres, 3 * Ns, h.data(), s))) return rc;
    for (int l = 0; l < Ns; ++l)
      blas_scale<double>(sol + (size_t)l * fs, h[3 * l + 2] > 0 ? 1.0 / sqrt(h[3 * l + 2]) : 0.0, 0.0, n, s);
    if ((rc = dw_pack(c, ip, Ns, sol, work, s))) return rc;
    ++*steps_done;
  }
  DW_CUDA(cudaStreamSynchronize(s));
  return DW_OK;
}

static int build_impl(dw_ctx* c, const dfl_params* p, const double* start, dfl_ctx* d, dfl_info* info) {
  const Geom& g = c->g;
  const size_t V = c->V;
  const int Ns = p->Ns;
  cudaStream_t s = 0;
  auto t0 = std::chrono::steady_clock::now();
  int rc;
  if ((rc = build_tables(c, d))) return rc;

  // ---- inverse iteration (5.1) in the requested precision
  const int ip = p->iter_prec == DW_F64 ? DW_F64 : DW_F32;
  const size_t fb = dw_field_bytes(c, ip);
  void* work = nullptr;
  void* tmp = nullptr;
  DW_CUDA(cudaMalloc(&work, fb * Ns));
  DW_CUDA(cudaMalloc(&tmp, fb));
  struct Free { void* a; void* b; ~Free() { if (a) cudaFree(a); if (b) cudaFree(b); } } guard{work, tmp};
  if ((rc = dw_pack(c, ip, Ns, start, work, s))) return rc;
  const size_t n = V * 12;
  std::vector<double> h(3);
  const bool use_net = p->net_weights != nullptr;
  if (use_net && (ip != DW_F32 || p->net_channels != 16 || p->net_k0 < 0 || p->net_k0 > p->n_inv)) {
    dw_set_error("deflation_build: the network needs iter_prec DW_F32, 16 channels and 0 <= net_k0 <= n_inv");
    return DW_EINVAL;
  }
  // mean ||D psi_l|| / ||psi_l|| of the FP32 work fields, the relaxation measure of (5.2)
  auto rho_measure = [&](const float* fields, double* out) -> int {
    double sum = 0;
    for (int l = 0; l < Ns; ++l) {
      const float* f = fields + (size_t)l * 24 * V;
      dirac_full<float>(c, f, (float*)tmp, s);
      blas_dot<float>(c, (float*)tmp, (float*)tmp, n, c->d_red + 65536, s);
      blas_dot<float>(c, f, f, n, c->d_red + 65536 + 3, s);
      double hh[6];
      int e = sync_read(c, c->d_red + 65536, 6, hh, s);
      if (e) return e;
      sum += sqrt(hh[2] / hh[5]);
    }
    *out = sum / Ns;
    return DW_OK;
  };
  int learned = 0;
  double rho_in = 0, rho_out = 0;
  const int n_first = use_net ? p->net_k0 : p->n_inv;
  for (int it = 0; it < n_first; ++it)
    for (int l = 0; l < Ns; ++l) {
      if (ip == DW_F64) {
        double* w = (double*)work + (size_t)l * 24 * V;
        if ((rc = sap_apply<double>(c, p->ncy, p->nmr, w, (double*)tmp, s))) return rc;
        blas_dot<double>(c, (double*)tmp, (double*)tmp, n, c->d_red + 65536, s);
        if ((rc = sync_read(c, c->d_red + 65536, 3, h.data(), s))) return rc;
        blas_convert<double, double>((double*)tmp, w, 1.0 / sqrt(h[2]), n, s);
      } else {
        float* w = (float*)work + (size_t)l * 24 * V;
        if ((rc = sap_apply<float>(c, p->ncy, p->nmr, w, (float*)tmp, s))) return rc;
        blas_dot<float>(c, (float*)tmp, (float*)tmp, n, c->d_red + 65536, s);
        if ((rc = sync_read(c, c->d_red + 65536, 3, h.data(), s))) return rc;
        blas_convert<float, float>((float*)tmp, w, 1.0 / sqrt(h[2]), n, s);
      }
    }
  if (use_net) {
    // learned generation: network on the fields after net_k0 plain steps, judged by (5.2)
    if ((rc = rho_measure((const float*)work, &rho_in))) return rc;
    float* out = nullptr;
    DW_CUDA(cudaMalloc(&out, fb * Ns));
    struct F1 { void* p; ~F1() { if (p) cudaFree(p); } } g2{out};
    if ((rc = ptnet_forward(c, p->net_channels, p->net_weights, Ns, work, out, s))) return rc;
    for (int l = 0; l < Ns; ++l) {
      float* f = out + (size_t)l * 24 * V;
      blas_dot<float>(c, f, f, n, c->d_red + 65536, s);
      if ((rc = sync_read(c, c->d_red + 65536, 3, h.data(), s))) return rc;
      blas_scale<float>(f, h[2] > 0 ? 1.0 / sqrt(h[2]) : 0.0, 0.0, n, s);
    }
    if ((rc = rho_measure(out, &rho_out))) return rc;
    if (std::isfinite(rho_out) && rho_out <= p->net_judge * rho_in) {
      learned = 1;
      DW_CUDA(cudaMemcpyAsync(work, out, fb * Ns, cudaMemcpyDeviceToDevice, s));
    } else {
      // fallback: the plain procedure finishes the generation
      for (int it = p->net_k0; it < p->n_inv; ++it)
        for (int l = 0; l < Ns; ++l) {
          float* w = (float*)work + (size_t)l * 24 * V;
          if ((rc = sap_apply<float>(c, p->ncy, p->nmr, w, (float*)tmp, s))) return rc;
          blas_dot<float>(c, (float*)tmp, (float*)tmp, n, c->d_red + 65536, s);
          if ((rc = sync_read(c, c->d_red + 65536, 3, h.data(), s))) return rc;
          blas_convert<float, float>((float*)tmp, w, 1.0 / sqrt(h[2]), n, s);
        }
      if ((rc = rho_measure((const float*)work, &rho_out))) return rc;
    }
  }
  // ---- bootstrapped inverse iteration (Section 5.3): after the plain steps, boot_steps further
  // steps psi_l <- "D^{-1}" psi_l in which D^{-1} is the deflated SAP-GCR solver on the subspace of
  // the current fields, stopped at the loose relative tolerance boot_tol (or boot_nmx GCR steps)
  int boot_steps_done = 0, boot_gcr = 0;
  if (p->boot_steps > 0) {
    if ((rc = bootstrap_steps(c, p, work, ip, &boot_steps_done, &boot_gcr))) return rc;
  }
  // the relaxation measure (5.2) of the generated fields (FP32 fields only; the network path has it)
  if (!use_net && ip == DW_F32 && (rc = rho_measure((const float*)work, &rho_out))) return rc;
  // ---- block Gram-Schmidt in FP64
  DW_CUDA(cudaMalloc(&d->basis64, (size_t)Ns * 24 * V * sizeof(double)));
  if (ip == DW_F64) DW_CUDA(cudaMemcpyAsync(d->basis64, work, fb * Ns, cudaMemcpyDeviceToDevice, s));
  else
    for (int l = 0; l < Ns; ++l)
      field_convert<float, double>((const float*)work + (size_t)l * 24 * V, d->basis64 + (size_t)l * 24 * V, 1.0,
                                   V, s);
  int* d_flag = (int*)(c->d_count + 40);
  DW_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
  block_gs_kernel<<<d->Nb, 256, 0, s>>>(g, d->d_sub, d->nsub, Ns, d->basis64, d_flag); dw_note_launch();
  int flag = 0;
  DW_CUDA(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  DW_CUDA(cudaStreamSynchronize(s));
  if (flag) { dw_set_error("deflation_build: rank loss in the block Gram-Schmidt"); return DW_EINVAL; }
  if (p->basis_prec == DW_BF16) {
    DW_CUDA(cudaMalloc(&d->basis16, (size_t)Ns * 3 * V * sizeof(uint4)));
    size_t tot = V * Ns;
    quantize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(V, Ns, d->basis64, d->basis16); dw_note_launch();
  }
  // ---- A.3 input: restriction coefficients (phi^L_k, psi_l) of the generated fields on the even blocks
  {
    const size_t ne = (size_t)d->Ne * Ns;
    d->graw.assign((size_t)Ns * ne, cd(0.0, 0.0));
    double* cfull;
    DW_CUDA(cudaMalloc(&cfull, (size_t)d->N * 2 * sizeof(double)));
    double* f64 = nullptr;
    if (ip == DW_F32) DW_CUDA(cudaMalloc(&f64, fb * 2));
    std::vector<double> hc((size_t)d->N * 2);
    for (int l = 0; l < Ns; ++l) {
      const double* src;
      if (ip == DW_F64) src = (const double*)work + (size_t)l * 24 * V;
      else {
        field_convert<float, double>((const float*)work + (size_t)l * 24 * V, f64, 1.0, V, s);
        src = f64;
      }
      restrict_kernel<double><<<d->Nb, 128, 0, s>>>(g, d->d_sub, d->nsub, Ns, d->basis64, nullptr, src, cfull, 1,
                                                    0, 0); dw_note_launch();
      DW_CUDA(cudaMemcpyAsync(hc.data(), cfull, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      DW_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i < d->Ne; ++i)
        for (int k = 0; k < Ns; ++k) {
          size_t o = ((size_t)d->hlist0[i] * Ns + k) * 2;
          d->graw[(size_t)l * ne + (size_t)i * Ns + k] = cd(hc[o], hc[o + 1]);
        }
    }
    cudaFree(cfull);
    if (f64) cudaFree(f64);
  }
  auto t1 = std::chrono::steady_clock::now();
  if ((rc = little_setup(c, d, nullptr))) return rc;
  drop_basis64(d);
  auto t2 = std::chrono::steady_clock::now();
  if (info) {
    info->seconds = std::chrono::duration<double>(t2 - t0).count();
    info->seconds_little = std::chrono::duration<double>(t2 - t1).count();
    info->max_block_cond = d->max_cond;
    info->Nb = d->Nb;
    info->N = d->N;
    info->learned_used = learned;
    info->rho_in = rho_in;
    info->rho_out = rho_out;
    info->boot_steps = boot_steps_done;
    info->boot_gcr_steps = boot_gcr;
  }
  return d->illcond ? DW_ILLCOND : DW_OK;
}

// a deflation context for operator c with the block geometry of p (validated)
static int dfl_alloc(dw_ctx* c, const dfl_params* p, dfl_ctx** out) {
  *out = nullptr;
  if (p->Ns < 1 || p->Ns > NSMAX || p->n_inv < 0 || p->ncy < 0 || p->nmr < 0 || p->boot_steps < 0 ||
      (p->basis_prec != DW_BF16 && p->basis_prec != DW_F64)) {
    dw_set_error("deflation_build: Ns must be in 1..32, counts non-negative, basis_prec DW_BF16 or DW_F64");
    return DW_EINVAL;
  }
  dfl_ctx* d = new dfl_ctx();
  d->c = c;
  d->p = *p;
  d->p.net_weights = nullptr;
  d->Ns = p->Ns;
  d->Nb = 1;
  d->nsub = 1;
  for (int mu = 0; mu < 4; ++mu) {
    int b = p->bs[mu];
    if (b <= 0 || b % c->g.sb[mu] != 0 || c->p.L[mu] % b != 0 || (c->p.L[mu] / b) % 2 != 0) {
      delete d;
      dw_set_error("deflation_build: bs[mu] must be a multiple of the Schwarz block dividing L[mu] an even number of times");
      return DW_EINVAL;
    }
    d->bs[mu] = b;
    d->nb[mu] = c->p.L[mu] / b;
    d->Nb *= d->nb[mu];
    d->nsub *= b / c->g.sb[mu];
  }
  d->N = d->Nb * d->Ns;
  *out = d;
  return DW_OK;
}

extern "C" int deflation_build(dw_ctx* c, const dfl_params* p, const double* start, dfl_ctx** out, dfl_info* info) {
  if (!c || !p || !start || !out) { dw_set_error("deflation_build: null argument"); return DW_EINVAL; }
  *out = nullptr;
  if (int rc = dw_check_device(c, "deflation_build")) return rc;
  if (p->boot_steps > 0 && (!(p->boot_tol > 0) || p->boot_nmx < 0)) {
    dw_set_error("deflation_build: boot_tol must be positive and boot_nmx non-negative");
    return DW_EINVAL;
  }
  dfl_ctx* d = nullptr;
  int rc = dfl_alloc(c, p, &d);
  if (rc) return rc;
  rc = build_impl(c, p, start, d, info);
  if (rc < 0) { dfl_destroy(d); return rc; }
  *out = d;
  return rc;
}

static bool same_geometry(const dw_ctx* a, const dw_ctx* b) {
  for (int mu = 0; mu < 4; ++mu)
    if (a->p.L[mu] != b->p.L[mu] || a->p.sap_bs[mu] != b->p.sap_bs[mu]) return false;
  return true;
}

static void fill_info(dfl_ctx* d, dfl_info* info, double secs, double secs_little, int loaded) {
  if (!info) return;
  *info = dfl_info{};
  info->seconds = secs;
  info->seconds_little = secs_little;
  info->max_block_cond = d->max_cond;
  info->Nb = d->Nb;
  info->N = d->N;
  info->little_loaded = loaded;
}

extern "C" int dfl_retarget(const dfl_ctx* src, dw_ctx* c, dfl_ctx** out, dfl_info* info) {
  if (!src || !c || !out) { dw_set_error("dfl_retarget: null argument"); return DW_EINVAL; }
  *out = nullptr;
  if (int rc = dw_check_device(c, "dfl_retarget")) return rc;
  if (!same_geometry(src->c, c)) {
    dw_set_error("dfl_retarget: the operator has another lattice or Schwarz block size");
    return DW_EINVAL;
  }
  auto t0 = std::chrono::steady_clock::now();
  dfl_ctx* d = nullptr;
  int rc = dfl_alloc(c, &src->p, &d);
  if (rc) return rc;
  const size_t V = c->V, Ns = d->Ns;
  auto fail = [&](int r) { dfl_destroy(d); return r; };
  if ((rc = build_tables(c, d))) return fail(rc);
  cudaError_t e = cudaMalloc(&d->basis64, Ns * 24 * V * sizeof(double));
  if (e == cudaSuccess && src->basis64)
    e = cudaMemcpy(d->basis64, src->basis64, Ns * 24 * V * sizeof(double), cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && src->basis16) {
    e = cudaMalloc(&d->basis16, Ns * 3 * V * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(d->basis16, src->basis16, Ns * 3 * V * sizeof(uint4), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && !src->basis64) {
      dequantize_kernel<<<(unsigned)((V * Ns + 255) / 256), 256>>>(V, (int)Ns, d->basis16, d->basis64); dw_note_launch();
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return fail(dw_cuda_fail(e, "dfl_retarget"));
  d->graw = src->graw;
  if ((rc = little_setup(c, d, nullptr))) return fail(rc);
  drop_basis64(d);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  fill_info(d, info, secs, secs, 0);
  *out = d;
  return d->illcond ? DW_ILLCOND : DW_OK;
}

// checkpoint file layout: header, basis (BF16 units or FP64 field), A.3 coefficients, FP64 little operator
struct DflFileHeader {
  char magic[8];           // "DWDFL01\0"
  int L[4], sap_bs[4], bs[4];
  int Ns, basis_prec, antiperiodic, Ne;
  double m0, csw, cond_max;
  uint64_t gauge_hash;
  uint64_t V, n_graw, n_B;
};

extern "C" int dfl_save(const dfl_ctx* d, const char* path) {
  if (!d || !path) { dw_set_error("dfl_save: null argument"); return DW_EINVAL; }
  const dw_ctx* c = d->c;
  if (int rc = dw_check_device(c, "dfl_save")) return rc;
  DflFileHeader h{};
  memcpy(h.magic, "DWDFL01", 8);
  for (int mu = 0; mu < 4; ++mu) { h.L[mu] = c->p.L[mu]; h.sap_bs[mu] = c->p.sap_bs[mu]; h.bs[mu] = d->bs[mu]; }
  h.Ns = d->Ns;
  h.basis_prec = d->basis16 ? DW_BF16 : DW_F64;
  h.antiperiodic = c->p.antiperiodic;
  h.Ne = d->Ne;
  h.m0 = c->p.m0;
  h.csw = c->p.csw;
  h.cond_max = d->p.cond_max;
  h.gauge_hash = c->gauge_hash;
  h.V = (uint64_t)c->V;
  h.n_graw = d->graw.size();
  h.n_B = (uint64_t)d->Nb * 9 * d->Ns * d->Ns * 2;
  const size_t nbasis = d->basis16 ? (size_t)d->Ns * 3 * c->V * sizeof(uint4) : (size_t)d->Ns * 24 * c->V * sizeof(double);
  std::vector<unsigned char> basis(nbasis);
  std::vector<double> B(h.n_B);
  cudaError_t e = cudaMemcpy(basis.data(), d->basis16 ? (const void*)d->basis16 : (const void*)d->basis64, nbasis,
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(B.data(), d->B64, h.n_B * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return dw_cuda_fail(e, "dfl_save");
  FILE* f = fopen(path, "wb");
  if (!f) { dw_set_error(std::string("dfl_save: cannot open ") + path); return DW_EINVAL; }
  bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(basis.data(), 1, nbasis, f) == nbasis &&
            fwrite(d->graw.data(), sizeof(cd), d->graw.size(), f) == d->graw.size() &&
            fwrite(B.data(), sizeof(double), B.size(), f) == B.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) { dw_set_error(std::string("dfl_save: write error on ") + path); return DW_EINVAL; }
  return DW_OK;
}

extern "C" int dfl_load(dw_ctx* c, const char* path, dfl_ctx** out, dfl_info* info) {
  if (!c || !path || !out) { dw_set_error("dfl_load: null argument"); return DW_EINVAL; }
  *out = nullptr;
  if (int rc = dw_check_device(c, "dfl_load")) return rc;
  auto t0 = std::chrono::steady_clock::now();
  FILE* f = fopen(path, "rb");
  if (!f) { dw_set_error(std::string("dfl_load: cannot open ") + path); return DW_EINVAL; }
  struct Close { FILE* f; ~Close() { fclose(f); } } closer{f};
  DflFileHeader h{};
  if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "DWDFL01", 8) != 0) {
    dw_set_error("dfl_load: not a deflation subspace file");
    return DW_EINVAL;
  }
  for (int mu = 0; mu < 4; ++mu)
    if (h.L[mu] != c->p.L[mu] || h.sap_bs[mu] != c->p.sap_bs[mu]) {
      dw_set_error("dfl_load: the file belongs to another lattice or Schwarz block size");
      return DW_EINVAL;
    }
  dfl_params p{};
  for (int mu = 0; mu < 4; ++mu) p.bs[mu] = h.bs[mu];
  p.Ns = h.Ns;
  p.basis_prec = h.basis_prec;
  p.iter_prec = DW_F32;
  p.cond_max = h.cond_max;
  p.ncy = 4;
  p.nmr = 4;
  dfl_ctx* d = nullptr;
  int rc = dfl_alloc(c, &p, &d);
  if (rc) return rc;
  auto fail = [&](int r) { dfl_destroy(d); return r; };
  if ((rc = build_tables(c, d))) return fail(rc);
  const size_t V = c->V, Ns = d->Ns;
  if (h.V != (uint64_t)V || h.Ne != d->Ne || h.n_graw != (uint64_t)Ns * d->Ne * Ns ||
      h.n_B != (uint64_t)d->Nb * 9 * Ns * Ns * 2) {
    dw_set_error("dfl_load: inconsistent sizes in the file");
    return fail(DW_EINVAL);
  }
  const bool bf16 = h.basis_prec == DW_BF16;
  const size_t nbasis = bf16 ? Ns * 3 * V * sizeof(uint4) : Ns * 24 * V * sizeof(double);
  std::vector<unsigned char> basis(nbasis);
  std::vector<double> B(h.n_B);
  d->graw.resize(h.n_graw);
  if (fread(basis.data(), 1, nbasis, f) != nbasis || fread(d->graw.data(), sizeof(cd), h.n_graw, f) != h.n_graw ||
      fread(B.data(), sizeof(double), h.n_B, f) != h.n_B) {
    dw_set_error("dfl_load: file too short");
    return fail(DW_EINVAL);
  }
  cudaError_t e = cudaMalloc(&d->basis64, Ns * 24 * V * sizeof(double));
  if (e == cudaSuccess && bf16) {
    e = cudaMalloc(&d->basis16, nbasis);
    if (e == cudaSuccess) e = cudaMemcpy(d->basis16, basis.data(), nbasis, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      dequantize_kernel<<<(unsigned)((V * Ns + 255) / 256), 256>>>(V, (int)Ns, d->basis16, d->basis64); dw_note_launch();
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    e = cudaMemcpy(d->basis64, basis.data(), nbasis, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(dw_cuda_fail(e, "dfl_load"));
  const bool same_op = h.gauge_hash == c->gauge_hash && h.m0 == c->p.m0 && h.csw == c->p.csw &&
                       h.antiperiodic == c->p.antiperiodic;
  if ((rc = little_setup(c, d, same_op ? B.data() : nullptr))) return fail(rc);
  drop_basis64(d);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  fill_info(d, info, secs, secs, same_op ? 1 : 0);
  *out = d;
  return d->illcond ? DW_ILLCOND : DW_OK;
}
