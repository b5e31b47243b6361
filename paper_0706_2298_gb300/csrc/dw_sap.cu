// Schwarz alternating procedure M_sap (Section 6.1; Section 5.3 uses it as
// the approximate inverse of the inverse iteration (5.1)).
//
//   xi = 0, r = rho; ncy times, for colour in (black, white):
//     for every block L of the colour: delta_L = MR_nmr(D^_L) applied to r|_L
//     xi += delta, r = rho - D xi
//
// GPU form.  One CTA per block of the current colour (blocks of one colour
// never touch).  The CTA keeps the block's even-odd MR iteration on chip:
//   * residual r|_L is read once; its boundary sites first receive the
//     change caused by the other colour's last correction (halo hops of
//     delta from the neighbouring blocks), so r = rho - D xi is maintained
//     exactly without a global operator application;
//   * r^_e = b_e - D_eo A_oo^{-1} b_o, then nmr MR steps
//         p = (A_ee - D_eo A_oo^{-1} D_oe) r^_e,  alpha = (p, r^)/|p|^2  (block reduction),
//         x_e += alpha r^_e,  r^_e -= alpha p
//     with r^_e and the odd intermediate in shared memory;
//   * odd reconstruction x_o = A_oo^{-1}(b_o - D_oe x_e);
//   * the new block residual is (r^_e, 0) exactly; it, the correction delta
//     and xi += delta are written back.
// Links and the clover term are read through the read-only cache.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <type_traits>

#include "dw_common.cuh"

namespace {

template <int MU, typename T, int SHV>
DW_D void inblock_dir(const Geom& g, const SiteRef& s, long long i, const uint16_t* nbe,
                      const T* __restrict__ links, const cplx<T>* sm, cplx<T>* acc) {
  const size_t V = g.V;
  SU3<T> U;
  cplx<T> p[12];
  uint16_t e = nbe[2 * MU];
  if (!(e >> 15)) {
    int hn = e & 0x7fff;
    load_link(links, V, MU, i, U);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = sm[k * SHV + hn];
    hop_acc<MU, -1, false>(acc, p, U, T(1));
  }
  e = nbe[2 * MU + 1];
  if (!(e >> 15)) {
    int hn = e & 0x7fff;
    load_link(links, V, MU, site_index(g, s.b, 1 - s.p, hn), U);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = sm[k * SHV + hn];
    hop_acc<MU, +1, true>(acc, p, U, T(1));
  }
}
template <typename T, int SHV>
DW_D void inblock_hops(const Geom& g, const SiteRef& s, long long i, const uint16_t* nbe,
                       const T* __restrict__ links, const cplx<T>* sm, cplx<T>* acc) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  inblock_dir<0, T, SHV>(g, s, i, nbe, links, sm, acc);
  inblock_dir<1, T, SHV>(g, s, i, nbe, links, sm, acc);
  inblock_dir<2, T, SHV>(g, s, i, nbe, links, sm, acc);
  inblock_dir<3, T, SHV>(g, s, i, nbe, links, sm, acc);
}

// acc += hops of a global field that cross the block boundary
template <int MU, typename T>
DW_D void halo_dir(const Geom& g, const SiteRef& s, long long i, const uint16_t* nbe,
                   const T* __restrict__ links, const T* __restrict__ f, cplx<T>* acc) {
  const size_t V = g.V;
  SU3<T> U;
  cplx<T> p[12];
  bool cr;
  if (nbe[2 * MU] >> 15) {
    long long j = neighbour(g, s, 2 * MU, &cr);
    T sg = time_wrap(g, s, 2 * MU) ? T(-1) : T(1);
    load_link(links, V, MU, i, U);
    load_site_rw<T, 12>(f, V, j, p);
    hop_acc<MU, -1, false>(acc, p, U, sg);
  }
  if (nbe[2 * MU + 1] >> 15) {
    long long j = neighbour(g, s, 2 * MU + 1, &cr);
    T sg = time_wrap(g, s, 2 * MU + 1) ? T(-1) : T(1);
    load_link(links, V, MU, j, U);
    load_site_rw<T, 12>(f, V, j, p);
    hop_acc<MU, +1, true>(acc, p, U, sg);
  }
}
template <typename T>
DW_D void halo_add(const Geom& g, const SiteRef& s, long long i, const uint16_t* nbe, const T* __restrict__ links,
                   const T* __restrict__ f, cplx<T>* b) {
  cplx<T> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  halo_dir<0>(g, s, i, nbe, links, f, acc);
  halo_dir<1>(g, s, i, nbe, links, f, acc);
  halo_dir<2>(g, s, i, nbe, links, f, acc);
  halo_dir<3>(g, s, i, nbe, links, f, acc);
  // r - D delta on the boundary: D contributes -1/2 * hops
#pragma unroll
  for (int k = 0; k < 12; ++k) b[k] += T(0.5) * acc[k];
}

// sum over the lanes of a warp that hold block threads (SHV < 32: only SHV lanes exist)
template <int SHV>
DW_D double warp_sum(double v) {
  constexpr unsigned mask = SHV >= 32 ? 0xffffffffu : ((1u << SHV) - 1u);
#pragma unroll
  for (int o = (SHV >= 32 ? 16 : SHV / 2); o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

template <typename T, int SHV>
__global__ void __launch_bounds__(SHV) sap_block_kernel(Geom g, const T* __restrict__ links,
                                                        const T* __restrict__ clov, const T* __restrict__ clovinv,
                                                        const int* __restrict__ blocks, const T* rsrc, T* rdst,
                                                        const T* dprev, T* dout, T* xi, int first, int nmr) {
  constexpr int NW = (SHV + 31) / 32;
  extern __shared__ __align__(16) unsigned char sap_smem[];
  cplx<T>* s_r = reinterpret_cast<cplx<T>*>(sap_smem);   // r^_e
  cplx<T>* s_t = s_r + 12 * SHV;                          // odd intermediate, later x_e
  cplx<T>* s_b = s_t + 12 * SHV;                          // b_o (source on odd sites)
  __shared__ double s_red[3][NW];
  const size_t V = g.V;
  const int h = threadIdx.x;
  const int b = blocks[blockIdx.x];
  SiteRef se = {b, 0, h}, so = {b, 1, h};
  const long long ie = site_index(g, b, 0, h), io = site_index(g, b, 1, h);
  uint16_t nbe_e[8], nbe_o[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    nbe_e[d] = __ldg(g.nbtab + (h << 3) + d);
    nbe_o[d] = __ldg(g.nbtab + ((SHV + h) << 3) + d);
  }
  cplx<T> v[12], w[12], acc[12];
  // ---- residual with halo correction
  load_site_rw<T, 12>(rsrc, V, io, v);
  if (dprev) halo_add(g, so, io, nbe_o, links, dprev, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) s_b[k * SHV + h] = v[k];
  clover_apply(clovinv, V, io, v, w);                       // A_oo^{-1} b_o
#pragma unroll
  for (int k = 0; k < 12; ++k) s_t[k * SHV + h] = w[k];
  load_site_rw<T, 12>(rsrc, V, ie, v);
  if (dprev) halo_add(g, se, ie, nbe_e, links, dprev, v);
  __syncthreads();
  inblock_hops<T, SHV>(g, se, ie, nbe_e, links, s_t, acc);  // r^_e = b_e - D_eo A^{-1} b_o
  cplx<T> x[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[k] += T(0.5) * acc[k];
    s_r[k * SHV + h] = v[k];
    x[k] = {T(0), T(0)};
  }
  __syncthreads();
  // ---- minimal residual steps on the even-odd block operator
  for (int it = 0; it < nmr; ++it) {
    inblock_hops<T, SHV>(g, so, io, nbe_o, links, s_r, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = T(-0.5) * acc[k];
    clover_apply(clovinv, V, io, acc, w);                   // A_oo^{-1} D_oe r^_e
    __syncthreads();                                        // all reads of s_t from the last step done
#pragma unroll
    for (int k = 0; k < 12; ++k) s_t[k * SHV + h] = w[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = s_r[k * SHV + h];
    clover_apply(clov, V, ie, v, w);                        // A_ee r^_e
    inblock_hops<T, SHV>(g, se, ie, nbe_e, links, s_t, acc);
    double pr = 0, pi = 0, pp = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      w[k] += T(0.5) * acc[k];                              // p = D^ r^
      pr += (double)w[k].re * v[k].re + (double)w[k].im * v[k].im;
      pi += (double)w[k].re * v[k].im - (double)w[k].im * v[k].re;
      pp += (double)w[k].re * w[k].re + (double)w[k].im * w[k].im;
    }
    pr = warp_sum<SHV>(pr); pi = warp_sum<SHV>(pi); pp = warp_sum<SHV>(pp);
    if ((h & 31) == 0) { s_red[0][h >> 5] = pr; s_red[1][h >> 5] = pi; s_red[2][h >> 5] = pp; }
    __syncthreads();
    pr = 0; pi = 0; pp = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) { pr += s_red[0][j]; pi += s_red[1][j]; pp += s_red[2][j]; }
    cplx<T> alpha = {T(0), T(0)};
    if (pp > 0) alpha = {(T)(pr / pp), (T)(pi / pp)};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      x[k] += alpha * v[k];
      v[k] -= alpha * w[k];
      s_r[k * SHV + h] = v[k];
    }
    __syncthreads();                                        // s_red reused, s_r complete
  }
  // ---- odd reconstruction x_o = A_oo^{-1}(b_o - D_oe x_e)
#pragma unroll
  for (int k = 0; k < 12; ++k) s_t[k * SHV + h] = x[k];
  __syncthreads();
  inblock_hops<T, SHV>(g, so, io, nbe_o, links, s_t, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = s_b[k * SHV + h] + T(0.5) * acc[k];
  clover_apply(clovinv, V, io, acc, w);                     // x_o
  // ---- outputs
  if (dout) {
    store_site<T, 12>(dout, V, ie, x);
    store_site<T, 12>(dout, V, io, w);
  }
  if (rdst) {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = s_r[k * SHV + h];
    store_site<T, 12>(rdst, V, ie, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = {T(0), T(0)};
    store_site<T, 12>(rdst, V, io, v);
  }
  if (!first) {
    load_site_rw<T, 12>(xi, V, ie, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] += v[k];
    load_site_rw<T, 12>(xi, V, io, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] += v[k];
  }
  store_site<T, 12>(xi, V, ie, x);
  store_site<T, 12>(xi, V, io, w);
}

// ============================================================================ staged FP32 kernel
// Same algorithm as sap_block_kernel, organised for throughput:
//  * the block's links are staged once into shared memory as full 3x3 matrices;
//  * 2*SHV threads: lanes 2h and 2h+1 (q = 0, 1) share the site pair h.  In the
//    hopping sums each thread projects onto spin q only: it loads half of each
//    neighbour spinor and does one SU(3) product per hop.  Two lane-pair shuffles
//    then regroup the sum by chirality: thread q owns chiral block q
//    (spins 2q, 2q+1 = components 6q..6q+5) of both sites, applies that 6x6 clover
//    block and keeps its share of the MR vectors.
// acc layout of a thread's hop share: [0..2] upper spin q, [3..5] lower spin 2+q, [6..8] lower spin 3-q

// z * (sgn) or z * (i sgn)
template <bool IMAG>
DW_D cplx<float> unit_mul(cplx<float> z, float sgn) {
  if (IMAG) return {-sgn * z.im, sgn * z.re};
  return {sgn * z.re, sgn * z.im};
}

template <int MU>
DW_D void half_hop_dir(const cplx<float>* __restrict__ sU, const cplx<float>* __restrict__ sm, int SHV, int lown,
                       int lnb_base, uint16_t ef, uint16_t eb, int q, cplx<float>* acc) {
  constexpr int NSITE_MUL = 2;
  (void)NSITE_MUL;
  const int NS = 2 * SHV;
  // e_mu psi_lo coefficient for spin q and the spin it takes from the lower half
  constexpr bool IM = (MU == 1 || MU == 3);
  const float sg = (MU == 0 || MU == 1) ? -1.f : (q ? 1.f : -1.f);
  const int lo = (MU == 0 || MU == 3) ? 2 + q : 3 - q;
  const int slot = (MU == 0 || MU == 3) ? 3 : 6;       // accumulator of the lower spin touched
  if (!(ef >> 15)) {                                   // forward: (1 - gamma) U(x) psi(x+mu)
    const int hn = ef & 0x7fff;
    cplx<float> hv[3], w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) hv[c] = sm[(3 * q + c) * SHV + hn] - unit_mul<IM>(sm[(3 * lo + c) * SHV + hn], sg);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx<float>* u = sU + (MU * 9 + 3 * a) * NS + lown;
      w[a] = u[0] * hv[0] + u[NS] * hv[1] + u[2 * NS] * hv[2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] += w[c];
      acc[slot + c] -= unit_mul<IM>(w[c], IM ? -sg : sg);   // S = -1, coefficient conj(e)
    }
  }
  if (!(eb >> 15)) {                                   // backward: (1 + gamma) U(x-mu)^+ psi(x-mu)
    const int hn = eb & 0x7fff;
    const int ln = lnb_base + hn;
    cplx<float> hv[3], w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) hv[c] = sm[(3 * q + c) * SHV + hn] + unit_mul<IM>(sm[(3 * lo + c) * SHV + hn], sg);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx<float>* u = sU + (MU * 9 + a) * NS + ln;
      w[a] = cmulc(u[0], hv[0]) + cmulc(u[3 * NS], hv[1]) + cmulc(u[6 * NS], hv[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] += w[c];
      acc[slot + c] += unit_mul<IM>(w[c], IM ? -sg : sg);
    }
  }
}

// hop share at a site -> this thread's chiral block (6 complex) of the full hopping sum
DW_D void staged_hops(const cplx<float>* sU, const cplx<float>* sm, int SHV, int p, int h, int q,
                      const uint16_t* nbe, cplx<float>* out6) {
  cplx<float> acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = {0.f, 0.f};
  const int lown = p * SHV + h, lnb = (1 - p) * SHV;
  half_hop_dir<0>(sU, sm, SHV, lown, lnb, nbe[0], nbe[1], q, acc);
  half_hop_dir<1>(sU, sm, SHV, lown, lnb, nbe[2], nbe[3], q, acc);
  half_hop_dir<2>(sU, sm, SHV, lown, lnb, nbe[4], nbe[5], q, acc);
  half_hop_dir<3>(sU, sm, SHV, lown, lnb, nbe[6], nbe[7], q, acc);
  // lower spin 2+q: own slot 3 + partner's slot 6 (its 3-q' = 2+q)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float re = __shfl_xor_sync(0xffffffffu, acc[6 + c].re, 1);
    float im = __shfl_xor_sync(0xffffffffu, acc[6 + c].im, 1);
    acc[3 + c] += cplx<float>{re, im};
  }
  // thread q holds spins q (upper) and 2+q (lower); chiral block q needs spins 2q, 2q+1:
  // q = 0 keeps spin 0 and receives spin 1; q = 1 keeps spin 3 and receives spin 2
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<float> send = q ? acc[c] : acc[3 + c];          // q=1 sends spin 1, q=0 sends spin 2
    float re = __shfl_xor_sync(0xffffffffu, send.re, 1);
    float im = __shfl_xor_sync(0xffffffffu, send.im, 1);
    if (q == 0) { out6[c] = acc[c]; out6[3 + c] = {re, im}; }
    else        { out6[c] = {re, im}; out6[3 + c] = acc[3 + c]; }
  }
}

DW_D void clover_block(const float* __restrict__ cl, size_t V, long long i, int q, const cplx<float>* x,
                       cplx<float>* y) {
  cplx<float> s[18];
  load_site<float, 18>(cl + (size_t)36 * V * q, V, i, s);
  herm6_mul(s, x, y);
}

template <int SHV>
__global__ void __launch_bounds__(2 * SHV, 2) sap_staged_kernel(Geom g, const float* __restrict__ links,
                                                                const float* __restrict__ clov,
                                                                const float* __restrict__ clovinv,
                                                                const int* __restrict__ blocks, const float* rsrc0,
                                                                float* rdst0, const float* dprev0, float* dout0,
                                                                float* xi0, int first, int nmr, int nrhs,
                                                                size_t fstride) {
  constexpr int NT = 2 * SHV, NS = 2 * SHV, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char sap_smem[];
  cplx<float>* sU = reinterpret_cast<cplx<float>*>(sap_smem);   // [4][9][NS]
  cplx<float>* s_r = sU + 36 * NS;                                // [12][SHV] even field
  cplx<float>* s_t = s_r + 12 * SHV;                              // [12][SHV] odd field, later x_e
  cplx<float>* s_b = s_t + 12 * SHV;                              // [12][SHV] b_o
  __shared__ float s_red[3][NW];
  const size_t V = g.V;
  const int t = threadIdx.x, h = t >> 1, q = t & 1;
  const int b = blocks[blockIdx.x];
  const long long base = (long long)b << g.lsvol;
  const long long ie = base + h, io = base + SHV + h;
  // ---- stage the block's links (full matrices)
  for (int idx = t; idx < 4 * NS; idx += NT) {
    const int mu = idx / NS, l = idx - mu * NS;
    SU3<float> U;
    load_link(links, V, mu, base + l, U);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) sU[(mu * 9 + 3 * a + c) * NS + l] = U.m[a][c];
  }
  uint16_t nbe_e[8], nbe_o[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    nbe_e[d] = __ldg(g.nbtab + (h << 3) + d);
    nbe_o[d] = __ldg(g.nbtab + ((SHV + h) << 3) + d);
  }
  // the staged links serve every right-hand side of the batch
  for (int rhs = 0; rhs < nrhs; ++rhs) {
  const size_t fo = (size_t)rhs * fstride;
  const float* rsrc = rsrc0 + fo;
  float* rdst = rdst0 ? rdst0 + fo : nullptr;
  const float* dprev = dprev0 ? dprev0 + fo : nullptr;
  float* dout = dout0 ? dout0 + fo : nullptr;
  float* xi = xi0 + fo;
  // ---- residual with halo correction: q = 0 takes the even site, q = 1 the odd site
  {
    cplx<float> v[12];
    const long long i = q ? io : ie;
    load_site_rw<float, 12>(rsrc, V, i, v);
    if (dprev) {
      SiteRef sr = {b, q, h};
      halo_add(g, sr, i, q ? nbe_o : nbe_e, links, dprev, v);
    }
    cplx<float>* dst = q ? s_b : s_r;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k * SHV + h] = v[k];
  }
  __syncthreads();
  cplx<float> v6[6], w6[6], h6[6], x6[6];
  // t_o = A_oo^{-1} b_o  (chiral block q)
#pragma unroll
  for (int j = 0; j < 6; ++j) v6[j] = s_b[(6 * q + j) * SHV + h];
  clover_block(clovinv, V, io, q, v6, w6);
#pragma unroll
  for (int j = 0; j < 6; ++j) s_t[(6 * q + j) * SHV + h] = w6[j];
  __syncthreads();
  // r^_e = b_e - D_eo t_o = b_e + 1/2 hops
  staged_hops(sU, s_t, SHV, 0, h, q, nbe_e, h6);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    cplx<float> r = s_r[(6 * q + j) * SHV + h] + 0.5f * h6[j];
    s_r[(6 * q + j) * SHV + h] = r;
    x6[j] = {0.f, 0.f};
  }
  __syncthreads();
  for (int it = 0; it < nmr; ++it) {
    // t_o = A_oo^{-1} D_oe r^_e
    staged_hops(sU, s_r, SHV, 1, h, q, nbe_o, h6);
#pragma unroll
    for (int j = 0; j < 6; ++j) v6[j] = -0.5f * h6[j];
    clover_block(clovinv, V, io, q, v6, w6);
#pragma unroll
    for (int j = 0; j < 6; ++j) s_t[(6 * q + j) * SHV + h] = w6[j];
    __syncthreads();
    // p = A_ee r^ - D_eo t_o
#pragma unroll
    for (int j = 0; j < 6; ++j) v6[j] = s_r[(6 * q + j) * SHV + h];
    clover_block(clov, V, ie, q, v6, w6);
    staged_hops(sU, s_t, SHV, 0, h, q, nbe_e, h6);
    float pr = 0.f, pi = 0.f, pp = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      w6[j] += 0.5f * h6[j];
      pr += w6[j].re * v6[j].re + w6[j].im * v6[j].im;
      pi += w6[j].re * v6[j].im - w6[j].im * v6[j].re;
      pp += w6[j].re * w6[j].re + w6[j].im * w6[j].im;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pr += __shfl_xor_sync(0xffffffffu, pr, o);
      pi += __shfl_xor_sync(0xffffffffu, pi, o);
      pp += __shfl_xor_sync(0xffffffffu, pp, o);
    }
    if ((t & 31) == 0) { s_red[0][t >> 5] = pr; s_red[1][t >> 5] = pi; s_red[2][t >> 5] = pp; }
    __syncthreads();
    pr = 0.f; pi = 0.f; pp = 0.f;
#pragma unroll
    for (int j = 0; j < NW; ++j) { pr += s_red[0][j]; pi += s_red[1][j]; pp += s_red[2][j]; }
    cplx<float> alpha = {0.f, 0.f};
    if (pp > 0.f) alpha = {pr / pp, pi / pp};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x6[j] += alpha * v6[j];
      v6[j] -= alpha * w6[j];
      s_r[(6 * q + j) * SHV + h] = v6[j];
    }
    __syncthreads();
  }
  // x_o = A_oo^{-1}(b_o - D_oe x_e)
#pragma unroll
  for (int j = 0; j < 6; ++j) s_t[(6 * q + j) * SHV + h] = x6[j];
  __syncthreads();
  staged_hops(sU, s_t, SHV, 1, h, q, nbe_o, h6);
#pragma unroll
  for (int j = 0; j < 6; ++j) v6[j] = s_b[(6 * q + j) * SHV + h] + 0.5f * h6[j];
  clover_block(clovinv, V, io, q, v6, w6);   // w6 = x_o (block q)
  // ---- outputs: this thread's three float4 units (components 6q..6q+5) of each site
  float4* dv = reinterpret_cast<float4*>(dout);
  float4* rv = reinterpret_cast<float4*>(rdst);
  float4* xv = reinterpret_cast<float4*>(xi);
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const size_t pe = (size_t)(3 * q + u) * V + ie, po = (size_t)(3 * q + u) * V + io;
    float4 xe = pack_unit(x6 + 2 * u), xo = pack_unit(w6 + 2 * u);
    if (dout) { dv[pe] = xe; dv[po] = xo; }
    if (rdst) {
      cplx<float> r2[2] = {s_r[(6 * q + 2 * u) * SHV + h], s_r[(6 * q + 2 * u + 1) * SHV + h]};
      rv[pe] = pack_unit(r2);
      rv[po] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!first) {
      float4 a = xv[pe], c = xv[po];
      xe.x += a.x; xe.y += a.y; xe.z += a.z; xe.w += a.w;
      xo.x += c.x; xo.y += c.y; xo.z += c.z; xo.w += c.w;
    }
    xv[pe] = xe;
    xv[po] = xo;
  }
  __syncthreads();   // shared buffers are reused by the next right-hand side
  }
}

template <int SHV>
bool launch_sap_staged(dw_ctx* c, int colour, const float* rsrc, float* rdst, const float* dprev, float* dout,
                       float* xi, int first, int nmr, cudaStream_t st, int nrhs = 1) {
  constexpr size_t smem = (36 * 2 * SHV + 3 * 12 * SHV) * sizeof(cplx<float>);
  static int state = 0;   // 0 unknown, 1 ok, -1 unavailable
  if (state == 0) {
    cudaError_t e = cudaFuncSetAttribute(sap_staged_kernel<SHV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    state = e == cudaSuccess ? 1 : -1;
  }
  if (state < 0) return false;
  const int* list = c->d_colour_list + (colour ? c->ncolour[0] : 0);
  sap_staged_kernel<SHV><<<c->ncolour[colour], 2 * SHV, smem, st>>>(c->g, (const float*)c->links[DW_F32],
                                                                   (const float*)c->clov[DW_F32],
                                                                   (const float*)c->clovinv[DW_F32], list, rsrc,
                                                                   rdst, dprev, dout, xi, first, nmr, nrhs,
                                                                   (size_t)c->V * 24); dw_note_launch();
  return true;
}

template <typename T, int SHV>
void launch_sap(dw_ctx* c, int colour, const T* rsrc, T* rdst, const T* dprev, T* dout, T* xi, int first, int nmr,
                cudaStream_t st) {
  constexpr int P = prec_of<T>();
  const int* list = c->d_colour_list + (colour ? c->ncolour[0] : 0);
  constexpr size_t smem = 3 * 12 * SHV * sizeof(cplx<T>);
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaFuncSetAttribute(sap_block_kernel<T, SHV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  sap_block_kernel<T, SHV><<<c->ncolour[colour], SHV, smem, st>>>(c->g, (const T*)c->links[P], (const T*)c->clov[P],
                                                              (const T*)c->clovinv[P], list, rsrc, rdst, dprev,
                                                              dout, xi, first, nmr); dw_note_launch();
}

}  // namespace

static dw_ctx* g_tune_ctx = nullptr;   // context whose autotuned choice applies to the current call
static bool use_staged() {
  const char* e = getenv("DW_SAP_STAGED");
  if (e) return e[0] != '0';
  return g_tune_ctx ? g_tune_ctx->tune_sap_staged != 0 : true;
}

template <typename T>
int sap_apply(dw_ctx* c, int ncy, int nmr, const T* rho, T* xi, cudaStream_t st) {
  g_tune_ctx = c;
  constexpr int P = prec_of<T>();
  size_t bytes = dw_field_bytes(c, P);
  if (!c->sap_r[P]) DW_CUDA(cudaMalloc(&c->sap_r[P], bytes * (P == DW_F32 && c->sap_cap > 1 ? c->sap_cap : 1)));
  if (!c->sap_d[P]) DW_CUDA(cudaMalloc(&c->sap_d[P], bytes * (P == DW_F32 && c->sap_cap > 1 ? c->sap_cap : 1)));
  if (ncy <= 0) {
    DW_CUDA(cudaMemsetAsync(xi, 0, bytes, st));
    return DW_OK;
  }
  T* r = (T*)c->sap_r[P];
  T* d = (T*)c->sap_d[P];
  for (int cy = 0; cy < ncy; ++cy)
    for (int col = 0; col < 2; ++col) {
      bool last = (cy == ncy - 1 && col == 1);
      const T* rsrc = cy == 0 ? rho : r;
      T* rdst = last ? nullptr : r;
      const T* dprev = (cy == 0 && col == 0) ? nullptr : d;
      T* dout = last ? nullptr : d;
      int first = cy == 0;
      if (std::is_same<T, float>::value && use_staged()) {
        bool ok = false;
        const float* rs = (const float*)rsrc; float* rd = (float*)rdst; const float* dp = (const float*)dprev;
        float* dd = (float*)dout; float* xx = (float*)xi;
        switch (c->g.shv) {
          case 16: ok = launch_sap_staged<16>(c, col, rs, rd, dp, dd, xx, first, nmr, st); break;
          case 32: ok = launch_sap_staged<32>(c, col, rs, rd, dp, dd, xx, first, nmr, st); break;
          case 64: ok = launch_sap_staged<64>(c, col, rs, rd, dp, dd, xx, first, nmr, st); break;
          case 128: ok = launch_sap_staged<128>(c, col, rs, rd, dp, dd, xx, first, nmr, st); break;
          default: break;
        }
        if (ok) continue;
      }
      switch (c->g.shv) {
        case 8: launch_sap<T, 8>(c, col, rsrc, rdst, dprev, dout, xi, first, nmr, st); break;
        case 16: launch_sap<T, 16>(c, col, rsrc, rdst, dprev, dout, xi, first, nmr, st); break;
        case 32: launch_sap<T, 32>(c, col, rsrc, rdst, dprev, dout, xi, first, nmr, st); break;
        case 64: launch_sap<T, 64>(c, col, rsrc, rdst, dprev, dout, xi, first, nmr, st); break;
        case 128: launch_sap<T, 128>(c, col, rsrc, rdst, dprev, dout, xi, first, nmr, st); break;
        default:
          dw_set_error("sap_precondition: unsupported Schwarz block volume");
          return DW_EINVAL;
      }
    }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
// M_sap on nrhs FP32 fields at once (staged kernel; falls back to one field at a time)
int sap_apply_mrhs(dw_ctx* c, int ncy, int nmr, const float* rho, float* xi, int nrhs, cudaStream_t st) {
  g_tune_ctx = c;
  const size_t fb = dw_field_bytes(c, DW_F32);
  if (c->sap_cap < nrhs) {
    sap_graphs_free(c);   // captured graphs refer to the old workspace
    for (int P = 0; P < 2; ++P) {
      if (c->sap_r[P]) { cudaFree(c->sap_r[P]); c->sap_r[P] = nullptr; }
      if (c->sap_d[P]) { cudaFree(c->sap_d[P]); c->sap_d[P] = nullptr; }
    }
    DW_CUDA(cudaMalloc(&c->sap_r[DW_F32], fb * nrhs));
    DW_CUDA(cudaMalloc(&c->sap_d[DW_F32], fb * nrhs));
    c->sap_cap = nrhs;
  }
  const size_t fs = (size_t)c->V * 24;
  if (ncy <= 0) {
    DW_CUDA(cudaMemsetAsync(xi, 0, fb * nrhs, st));
    return DW_OK;
  }
  if (!use_staged() || c->g.shv < 16 || c->g.shv > 128) {
    for (int r = 0; r < nrhs; ++r) {
      int rc = sap_apply<float>(c, ncy, nmr, rho + r * fs, xi + r * fs, st);
      if (rc) return rc;
    }
    return DW_OK;
  }
  float* r = (float*)c->sap_r[DW_F32];
  float* d = (float*)c->sap_d[DW_F32];
  for (int cy = 0; cy < ncy; ++cy)
    for (int col = 0; col < 2; ++col) {
      bool last = (cy == ncy - 1 && col == 1);
      const float* rsrc = cy == 0 ? rho : r;
      float* rdst = last ? nullptr : r;
      const float* dprev = (cy == 0 && col == 0) ? nullptr : d;
      float* dout = last ? nullptr : d;
      bool ok = false;
      switch (c->g.shv) {
        case 16: ok = launch_sap_staged<16>(c, col, rsrc, rdst, dprev, dout, xi, cy == 0, nmr, st, nrhs); break;
        case 32: ok = launch_sap_staged<32>(c, col, rsrc, rdst, dprev, dout, xi, cy == 0, nmr, st, nrhs); break;
        case 64: ok = launch_sap_staged<64>(c, col, rsrc, rdst, dprev, dout, xi, cy == 0, nmr, st, nrhs); break;
        case 128: ok = launch_sap_staged<128>(c, col, rsrc, rdst, dprev, dout, xi, cy == 0, nmr, st, nrhs); break;
        default: break;
      }
      if (!ok) {
        dw_set_error("sap_apply_mrhs: staged kernel unavailable");
        return DW_EINVAL;
      }
    }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

// ---------------------------------------------------------------- CUDA graphs of M_sap
struct SapGraph {
  int uses = 0;
  cudaGraphExec_t exec = nullptr;
  int nodes = 0;
};
using SapKey = std::tuple<const void*, void*, int, int, int>;
using SapGraphMap = std::map<SapKey, SapGraph>;

void sap_graphs_free(dw_ctx* c) {
  if (!c->graph_cache) return;
  auto* m = static_cast<SapGraphMap*>(c->graph_cache);
  for (auto& kv : *m)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  delete m;
  c->graph_cache = nullptr;
}

static bool graphs_enabled() {
  const char* e = getenv("DW_GRAPH");
  return !(e && e[0] == '0');
}

int sap_apply_mrhs_graph(dw_ctx* c, int ncy, int nmr, const float* rho, float* xi, int nrhs, cudaStream_t st) {
  if (!graphs_enabled() || c->sap_cap < nrhs) return sap_apply_mrhs(c, ncy, nmr, rho, xi, nrhs, st);
  if (!c->graph_cache) c->graph_cache = new SapGraphMap();
  auto& m = *static_cast<SapGraphMap*>(c->graph_cache);
  SapGraph& gph = m[SapKey(rho, xi, nrhs, ncy, nmr)];
  if (!gph.exec) {
    if (gph.uses++ == 0) return sap_apply_mrhs(c, ncy, nmr, rho, xi, nrhs, st);   // first use: run directly
    if (!c->cap_stream) DW_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph;
    const long long n0 = dw_launch_count();
    DW_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = sap_apply_mrhs(c, ncy, nmr, rho, xi, nrhs, c->cap_stream);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (rc) return rc;
    if (e != cudaSuccess) return dw_cuda_fail(e, "cudaStreamEndCapture");
    gph.nodes = (int)(dw_launch_count() - n0);
    e = cudaGraphInstantiate(&gph.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { gph.exec = nullptr; return dw_cuda_fail(e, "cudaGraphInstantiate"); }
  }
  DW_CUDA(cudaGraphLaunch(gph.exec, st));
  for (int i = 0; i < gph.nodes; ++i) dw_note_launch();   // the graph's kernels
  return DW_OK;
}

// ---------------------------------------------------------------- autotuner
// Times the candidate launch shapes on this lattice with CUDA events (median of 5 after 2 warm-ups)
// and keeps the fastest: the multi-RHS D as one thread per (site, right-hand side) with the chunks
// interleaved, or one thread per site with 1, 2 or 3 right-hand sides per pass; the staged or
// generic FP32 Schwarz kernel.
extern "C" int dw_autotune(dw_ctx* c, int nrhs, char* report, size_t report_len) {
  if (!c || nrhs < 1 || nrhs > 64) { dw_set_error("dw_autotune: bad argument"); return DW_EINVAL; }
  const size_t fb = dw_field_bytes(c, DW_F32);
  float *x = nullptr, *y = nullptr;
  DW_CUDA(cudaMalloc(&x, fb * nrhs));
  cudaError_t e = cudaMalloc(&y, fb * nrhs);
  if (e != cudaSuccess) { cudaFree(x); return dw_cuda_fail(e, "cudaMalloc"); }
  cudaMemset(x, 0, fb * nrhs);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto time_it = [&](auto fn) {
    std::vector<float> ts;
    for (int it = 0; it < 7; ++it) {
      cudaEventRecord(a, 0);
      fn();
      cudaEventRecord(b, 0);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (it >= 2) ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
  };
  float td[4] = {0, 0, 0, 0};
  int best_r = 0;
  for (int rg = 0; rg <= 3; ++rg) {     // 0: one thread per (site, right-hand side), chunk-interleaved
    td[rg] = time_it([&] { dirac_mrhs<float>(c, x, y, nrhs, rg, 0); });
    if (td[rg] < td[best_r]) best_r = rg;
  }
  c->tune_rgroup = best_r;
  float ts[2] = {0, 0};
  const char* env = getenv("DW_SAP_STAGED");
  for (int st = 0; st < 2; ++st) {
    c->tune_sap_staged = st;
    if (!env) ts[st] = time_it([&] { sap_apply<float>(c, 1, 4, x, y, 0); });
  }
  c->tune_sap_staged = (env || ts[1] <= ts[0]) ? 1 : 0;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(x);
  cudaFree(y);
  if (report && report_len) {
    snprintf(report, report_len,
             "{\"nrhs\": %d, \"dirac_mrhs_ms\": {\"interleaved\": %.4f, \"1\": %.4f, \"2\": %.4f, \"3\": %.4f}, "
             "\"rgroup\": %d, "
             "\"sap_pass_ms\": {\"generic\": %.4f, \"staged\": %.4f}, \"sap_staged\": %d}",
             nrhs, td[0], td[1], td[2], td[3], best_r, ts[0], ts[1], c->tune_sap_staged);
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

template int sap_apply<float>(dw_ctx*, int, int, const float*, float*, cudaStream_t);
template int sap_apply<double>(dw_ctx*, int, int, const double*, double*, cudaStream_t);

extern "C" int sap_precondition(dw_ctx* c, int prec, int ncy, int nmr, int nrhs, const void* rho, void* xi,
                                void* stream) {
  if (!c || !rho || !xi || rho == xi || nrhs < 1 || nmr < 0 || (prec != DW_F64 && prec != DW_F32)) {
    dw_set_error("sap_precondition: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "sap_precondition")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = (size_t)c->V * 24;
  if (prec == DW_F32 && nrhs > 1) return sap_apply_mrhs(c, ncy, nmr, (const float*)rho, (float*)xi, nrhs, st);
  for (int r = 0; r < nrhs; ++r) {
    int rc = prec == DW_F64 ? sap_apply(c, ncy, nmr, (const double*)rho + r * n, (double*)xi + r * n, st)
                            : sap_apply(c, ncy, nmr, (const float*)rho + r * n, (float*)xi + r * n, st);
    if (rc) return rc;
  }
  return DW_OK;
}
