// Wilson-clover operator D (Section 2.1 operator) and its even-odd Schur
// complement A_ee - D_eo A_oo^{-1} D_oe, on packed fields.
//
// One thread per output site; 16-byte structure-of-arrays loads; links
// stored as two rows (third rebuilt in registers); spin projection with the
// chiral-basis (1 -+ gamma_mu) so that only 2x3 complex numbers go through
// each SU(3) multiply.  The kernel is HBM-bound: per site it moves the
// quark field (in + out), 4 links and the clover term once, with the
// neighbour re-reads served by L2 (block-major order keeps them close).
#include "dw_common.cuh"

#include <cstdio>
#include <cstdlib>
#include <mutex>

template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) dirac_full_kernel(Geom g, const T* __restrict__ links,
                                                         const T* __restrict__ clov, const T* __restrict__ in,
                                                         T* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  const size_t V = g.V;
  SiteRef s = decode(g, i);
  cplx<T> psi[12], y[12], acc[12];
  load_site<T, 12>(in, V, i, psi);
  clover_apply(clov, V, i, psi, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, i, links, in, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] -= T(0.5) * acc[k];
  store_site<T, 12>(out, V, i, y);
}

// Multi-RHS D with one thread per (site, right-hand side): the nrhs CTAs of one chunk of 128 sites
// are consecutive in launch order (blockIdx.x = chunk * nrhs + rhs), so the chunk's links and clover
// term come from HBM once and from L2 for the other right-hand sides (fields fstride reals apart).
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) dirac_interleaved_kernel(
    Geom g, const T* __restrict__ links, const T* __restrict__ clov, const T* __restrict__ in0, T* __restrict__ out0,
    int nrhs, size_t fstride) {
  const int r = blockIdx.x % nrhs;
  const long long i = (long long)(blockIdx.x / nrhs) * blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  const T* in = in0 + (size_t)r * fstride;
  T* out = out0 + (size_t)r * fstride;
  const size_t V = g.V;
  SiteRef s = decode(g, i);
  cplx<T> psi[12], y[12], acc[12];
  load_site<T, 12>(in, V, i, psi);
  clover_apply(clov, V, i, psi, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, i, links, in, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] -= T(0.5) * acc[k];
  store_site<T, 12>(out, V, i, y);
}

// t_o = A_oo^{-1} D_oe in_e   (odd sites; D_oe = -1/2 * hops)
template <typename T>
__global__ void __launch_bounds__(128) schur_odd_kernel(Geom g, const T* __restrict__ links,
                                                        const T* __restrict__ clovinv, const T* __restrict__ in,
                                                        T* __restrict__ t) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= g.V / 2) return;
  const size_t V = g.V;
  SiteRef s;
  s.b = (int)(tid >> g.lshv);
  s.p = 1;
  s.h = (int)(tid & (g.shv - 1));
  long long i = site_index(g, s.b, 1, s.h);
  cplx<T> acc[12], v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, i, links, in, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = T(-0.5) * acc[k];
  clover_apply(clovinv, V, i, acc, v);
  store_site<T, 12>(t, V, i, v);
}

// out_e = A_ee in_e - D_eo t_o ; out_o = 0
template <typename T>
__global__ void __launch_bounds__(128) schur_even_kernel(Geom g, const T* __restrict__ links,
                                                         const T* __restrict__ clov, const T* __restrict__ in,
                                                         const T* __restrict__ t, T* __restrict__ out) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= g.V / 2) return;
  const size_t V = g.V;
  SiteRef s;
  s.b = (int)(tid >> g.lshv);
  s.p = 0;
  s.h = (int)(tid & (g.shv - 1));
  long long i = site_index(g, s.b, 0, s.h);
  cplx<T> psi[12], y[12], acc[12];
  load_site<T, 12>(in, V, i, psi);
  clover_apply(clov, V, i, psi, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, i, links, t, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] += T(0.5) * acc[k];
  store_site<T, 12>(out, V, i, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] = {T(0), T(0)};
  store_site<T, 12>(out, V, site_index(g, s.b, 1, s.h), y);
}

// Even-odd preparation and reconstruction of D psi = eta (the Schur complement system
// (A_ee - D_eo A_oo^{-1} D_oe) psi_e = eta_e - D_eo A_oo^{-1} eta_o, psi_o = A_oo^{-1}(eta_o - D_oe psi_e)).
// t_o = A_oo^{-1} in_o on the odd sites
template <typename T>
__global__ void __launch_bounds__(128) clover_inv_odd_kernel(Geom g, const T* __restrict__ clovinv,
                                                             const T* __restrict__ in, T* __restrict__ t) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= g.V / 2) return;
  const size_t V = g.V;
  const int b = (int)(tid >> g.lshv), h = (int)(tid & (g.shv - 1));
  long long i = site_index(g, b, 1, h);
  cplx<T> x[12], y[12];
  load_site<T, 12>(in, V, i, x);
  clover_apply(clovinv, V, i, x, y);
  store_site<T, 12>(t, V, i, y);
}

// out_e = in_e - D_eo t_o = in_e + (1/2) hop(t) on the even sites, out_o = 0
template <typename T>
__global__ void __launch_bounds__(128) eo_rhs_kernel(Geom g, const T* __restrict__ links, const T* __restrict__ in,
                                                     const T* __restrict__ t, T* __restrict__ out) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= g.V / 2) return;
  const size_t V = g.V;
  SiteRef s;
  s.b = (int)(tid >> g.lshv);
  s.p = 0;
  s.h = (int)(tid & (g.shv - 1));
  long long i = site_index(g, s.b, 0, s.h);
  cplx<T> y[12], acc[12];
  load_site<T, 12>(in, V, i, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, i, links, t, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] += T(0.5) * acc[k];
  store_site<T, 12>(out, V, i, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] = {T(0), T(0)};
  store_site<T, 12>(out, V, site_index(g, s.b, 1, s.h), y);
}

// out_o = A_oo^{-1} (in_o - D_oe x_e) = A_oo^{-1} (in_o + (1/2) hop(x)) on the odd sites, out_e = x_e
template <typename T>
__global__ void __launch_bounds__(128) eo_reconstruct_kernel(Geom g, const T* __restrict__ links,
                                                             const T* __restrict__ clovinv, const T* __restrict__ in,
                                                             const T* __restrict__ x, T* __restrict__ out) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= g.V / 2) return;
  const size_t V = g.V;
  SiteRef s;
  s.b = (int)(tid >> g.lshv);
  s.p = 1;
  s.h = (int)(tid & (g.shv - 1));
  long long io = site_index(g, s.b, 1, s.h), ie = site_index(g, s.b, 0, s.h);
  cplx<T> y[12], acc[12], z[12];
  load_site<T, 12>(in, V, io, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {T(0), T(0)};
  hop_all(g, s, io, links, x, acc);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] += T(0.5) * acc[k];
  clover_apply(clovinv, V, io, y, z);
  store_site<T, 12>(out, V, io, z);
  load_site<T, 12>(x, V, ie, y);
  store_site<T, 12>(out, V, ie, y);
}

// Multi-RHS D: one thread per site applies D to all right-hand sides (fields stored one after the
// other, stride fstride reals).  RHS are processed R at a time; the links and clover of the site are
// loaded for each group but come from L1/L2 after the first, so HBM sees them once per site.
template <typename T, int R>
__global__ void __launch_bounds__(128) dirac_mrhs_kernel(Geom g, const T* __restrict__ links,
                                                         const T* __restrict__ clov, const T* __restrict__ in,
                                                         T* __restrict__ out, int nrhs, size_t fstride) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.V) return;
  const size_t V = g.V;
  SiteRef s = decode(g, i);
  for (int r0 = 0; r0 < nrhs; r0 += R) {
    const int nr = nrhs - r0 < R ? nrhs - r0 : R;
    cplx<T> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[r][k] = {T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int mu = d >> 1;
      bool cr;
      const long long j = neighbour(g, s, d, &cr);
      const T sg = time_wrap(g, s, d) ? T(-1) : T(1);
      SU3<T> U;
      load_link(links, V, mu, (d & 1) ? j : i, U);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < nr) {
          cplx<T> p[12];
          load_site<T, 12>(in + (size_t)(r0 + r) * fstride, V, j, p);
          switch (d) {
            case 0: hop_acc<0, -1, false>(acc[r], p, U, sg); break;
            case 1: hop_acc<0, +1, true>(acc[r], p, U, sg); break;
            case 2: hop_acc<1, -1, false>(acc[r], p, U, sg); break;
            case 3: hop_acc<1, +1, true>(acc[r], p, U, sg); break;
            case 4: hop_acc<2, -1, false>(acc[r], p, U, sg); break;
            case 5: hop_acc<2, +1, true>(acc[r], p, U, sg); break;
            case 6: hop_acc<3, -1, false>(acc[r], p, U, sg); break;
            default: hop_acc<3, +1, true>(acc[r], p, U, sg); break;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < nr) {
        cplx<T> psi[12], y[12];
        load_site<T, 12>(in + (size_t)(r0 + r) * fstride, V, i, psi);
        clover_apply(clov, V, i, psi, y);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] -= T(0.5) * acc[r][k];
        store_site<T, 12>(out + (size_t)(r0 + r) * fstride, V, i, y);
      }
    }
  }
}

template <typename T>
void dirac_mrhs(dw_ctx* c, const T* in, T* out, int nrhs, int rgroup, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  unsigned blocks = (unsigned)((c->V + 127) / 128);
  const size_t fs = (size_t)c->V * 24;
  const T* L = (const T*)c->links[P];
  const T* K = (const T*)c->clov[P];
  if (rgroup == 0) {
    const unsigned chunks = (unsigned)((c->V + 127) / 128);
    dirac_interleaved_kernel<T><<<chunks * (unsigned)nrhs, 128, 0, st>>>(c->g, L, K, in, out, nrhs, fs);
    dw_note_launch();
    return;
  }
  if (rgroup >= 3) { dirac_mrhs_kernel<T, 3><<<blocks, 128, 0, st>>>(c->g, L, K, in, out, nrhs, fs); dw_note_launch(); }
  else if (rgroup == 2) { dirac_mrhs_kernel<T, 2><<<blocks, 128, 0, st>>>(c->g, L, K, in, out, nrhs, fs); dw_note_launch(); }
  else { dirac_mrhs_kernel<T, 1><<<blocks, 128, 0, st>>>(c->g, L, K, in, out, nrhs, fs); dw_note_launch(); }
}
template void dirac_mrhs<float>(dw_ctx*, const float*, float*, int, int, cudaStream_t);
template void dirac_mrhs<double>(dw_ctx*, const double*, double*, int, int, cudaStream_t);

template <typename T>
void dirac_full(dw_ctx* c, const T* in, T* out, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  unsigned blocks = (unsigned)((c->V + 127) / 128);
  dirac_full_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clov[P], in, out); dw_note_launch();
}
template void dirac_full<float>(dw_ctx*, const float*, float*, cudaStream_t);
template void dirac_full<double>(dw_ctx*, const double*, double*, cudaStream_t);

// D on double-float fields with two threads per site (warps 2m and 2m+1 take the same 32
// sites): thread half q forms the spin-q component of every half-spinor projection, multiplies it
// by the link and adds it to spin q and to the lower spin it feeds; the two halves exchange their
// lower-spin partial sums through shared memory, and each applies rows 3q..3q+2 of both chiral
// clover blocks.  Half the arithmetic and registers per thread of dirac_full_kernel<dd>.
// s + e = a b for double-float a, b, exact up to the product of the low parts (Dekker's product of
// the leading parts by one FMA); s + e += a b with the leading part added by TwoSum and all errors
// gathered in e (compensated dot product, Ogita, Rump and Oishi 2005)
DW_D void dd2_first(float& s, float& e, dd a, dd b) {
  s = __fmul_rn(a.hi, b.hi);
  e = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -s)));
}
DW_D void dd2_acc(float& s, float& e, dd a, dd b) {
  const float h = __fmul_rn(a.hi, b.hi);
  const float l = __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.hi, b.hi, -h)));
  const float t = __fadd_rn(s, h);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(h, bb));
  s = t;
  e = __fadd_rn(e, __fadd_rn(err, l));
}
// o = U h (DAG: U^+ h) in double-float precision, each output component a compensated sum of its
// six real products (about 40% fewer FP32 operations than product-by-product double-float arithmetic)
template <bool DAG>
DW_D void su3_mul_dd2(const SU3<dd>& U, const cplx<dd>* h, cplx<dd>* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float sr, er, si, ei;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<dd> u = DAG ? U.m[c][a] : U.m[a][c];
      const dd ui = DAG ? -u.im : u.im;               // conj(U)^T for the adjoint
      if (c == 0) {
        dd2_first(sr, er, u.re, h[c].re);
        dd2_first(si, ei, u.re, h[c].im);
      } else {
        dd2_acc(sr, er, u.re, h[c].re);
        dd2_acc(si, ei, u.re, h[c].im);
      }
      dd2_acc(sr, er, -ui, h[c].im);
      dd2_acc(si, ei, ui, h[c].re);
    }
    o[a] = {dd_two_sum(sr, er), dd_two_sum(si, ei)};
  }
}

template <int MU, bool DAG>
DW_D void dd_half_hop(const dd* __restrict__ links, const dd* __restrict__ in, size_t V, long long j,
                      long long lk, int q, bool flip, cplx<dd>* au, cplx<dd>* al2, cplx<dd>* al3) {
  // lower spin feeding / fed by component q: 2 + q for mu = 0, 3; 3 - q for mu = 1, 2
  const int lo = (MU == 0 || MU == 3) ? 2 + q : 3 - q;
  SU3<dd> U;
  load_link(links, V, MU, lk, U);
  cplx<dd> pu[3], pl[3];
  const float4* P = reinterpret_cast<const float4*>(in);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    unpack_unit(__ldg(P + (size_t)(3 * q + c) * V + j), pu + c);
    unpack_unit(__ldg(P + (size_t)(3 * lo + c) * V + j), pl + c);
  }
  // v_q = e_mu-part of the lower spins: mu 0: -psi_lo; 1: -i psi_lo; 2: (q ? +1 : -1) psi_lo;
  // 3: (q ? +i : -i) psi_lo.  h = psi_q + S v_q with S = -1 forward (DAG = false), +1 backward.
  // S = +1 (DAG) or -1, sg = -1 (flip: antiperiodic wrap) or +1: products with them are sign flips
  cplx<dd> h[3], w[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<dd> v;
    if (MU == 0) v = -pl[c];
    else if (MU == 1) v = -ti(pl[c]);
    else if (MU == 2) v = q ? pl[c] : -pl[c];
    else v = q ? ti(pl[c]) : -ti(pl[c]);
    h[c] = DAG ? pu[c] + v : pu[c] - v;
  }
  su3_mul_dd2<DAG>(U, h, w);
  // the lower-spin image of w_q: mu 0: -w; 1: i w; 2: (q ? +w : -w); 3: (q ? -i w : i w)
  const bool neg_lower = (!DAG) != flip;               // S sg = -1
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    au[c] += flip ? -w[c] : w[c];
    cplx<dd> l;
    if (MU == 0) l = -w[c];
    else if (MU == 1) l = ti(w[c]);
    else if (MU == 2) l = q ? w[c] : -w[c];
    else l = q ? -ti(w[c]) : ti(w[c]);
    const cplx<dd> add = neg_lower ? -l : l;
    if (lo == 2) al2[c] += add; else al3[c] += add;
  }
}

// rows r0..r0+2 of one packed Hermitian 6x6 chiral block times x (6 components)
template <int R0>
DW_D void herm6_rows(const cplx<dd>* s, const cplx<dd>* x, cplx<dd>* y) {
  const dd d[6] = {s[0].re, s[0].im, s[1].re, s[1].im, s[2].re, s[2].im};
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] = d[R0 + r] * x[R0 + r];
  int k = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      if (i >= R0 && i < R0 + 3) y[i - R0] += s[k] * x[j];
      if (j >= R0 && j < R0 + 3) y[j - R0] += cmulc(s[k], x[i]);
      ++k;
    }
  }
}

__global__ void __launch_bounds__(128) dirac_dd_split_kernel(Geom g, const dd* __restrict__ links,
                                                             const dd* __restrict__ clov, const dd* __restrict__ in,
                                                             dd* __restrict__ out) {
  __shared__ cplx<dd> xch[2][3][64];          // lower-spin partials handed to the other half
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int q = w & 1, grp = w >> 1;           // warp-uniform half
  const int sl = grp * 32 + lane;              // site slot in the CTA (0..63)
  const long long i = (long long)blockIdx.x * 64 + sl;
  const bool valid = i < g.V;
  const size_t V = g.V;
  cplx<dd> au[3], a2[3], a3[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) { au[c] = {dd(0), dd(0)}; a2[c] = au[c]; a3[c] = au[c]; }
  if (valid) {
    const SiteRef s = decode(g, i);
    bool cr;
#define DD_DIR(MU)                                                                        \
    {                                                                                     \
      long long j = neighbour(g, s, 2 * MU, &cr);                                         \
      bool flip = time_wrap(g, s, 2 * MU);                                                \
      dd_half_hop<MU, false>(links, in, V, j, i, q, flip, au, a2, a3);                    \
      j = neighbour(g, s, 2 * MU + 1, &cr);                                               \
      flip = time_wrap(g, s, 2 * MU + 1);                                                 \
      dd_half_hop<MU, true>(links, in, V, j, j, q, flip, au, a2, a3);                     \
    }
    DD_DIR(0) DD_DIR(1) DD_DIR(2) DD_DIR(3)
#undef DD_DIR
  }
  // half q keeps lower spin 2 + q: hand the other lower spin to the partner half
#pragma unroll
  for (int c = 0; c < 3; ++c) xch[q][c][sl] = q ? a2[c] : a3[c];
  __syncthreads();
  if (!valid) return;
  cplx<dd> al[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) al[c] = (q ? a3[c] : a2[c]) + xch[1 - q][c][sl];
  // clover: rows 3q..3q+2 of both chiral blocks (block 0: spins 0, 1; block 1: spins 2, 3)
  cplx<dd> x[6], sblk[18], y0[3], y1[3];
  const float4* P = reinterpret_cast<const float4*>(in);
#pragma unroll
  for (int k = 0; k < 6; ++k) unpack_unit(__ldg(P + (size_t)k * V + i), x + k);
  load_site<dd, 18>(clov, V, i, sblk);
  if (q) herm6_rows<3>(sblk, x, y0); else herm6_rows<0>(sblk, x, y0);
#pragma unroll
  for (int k = 0; k < 6; ++k) unpack_unit(__ldg(P + (size_t)(6 + k) * V + i), x + k);
  load_site<dd, 18>(clov + 36 * V, V, i, sblk);
  if (q) herm6_rows<3>(sblk, x, y1); else herm6_rows<0>(sblk, x, y1);
  // out spin q (block 0 rows 3q..) and spin 2 + q (block 1 rows 3q..)
  float4* O = reinterpret_cast<float4*>(out);
  const dd hf = dd(0.5f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cplx<dd> u = y0[c] - hf * au[c];
    const cplx<dd> l = y1[c] - hf * al[c];
    O[(size_t)(3 * q + c) * V + i] = pack_unit(&u);
    O[(size_t)(3 * (2 + q) + c) * V + i] = pack_unit(&l);
  }
}

void dirac_full_dd(dw_ctx* c, const dd* in, dd* out, cudaStream_t st) {
  const char* e = getenv("DW_DD_SPLIT");
  if (e && e[0] == '0') {
    unsigned blocks = (unsigned)((c->V + 127) / 128);
    dirac_full_kernel<dd><<<blocks, 128, 0, st>>>(c->g, (const dd*)c->links_dd, (const dd*)c->clov_dd, in, out);
  } else {
    unsigned blocks = (unsigned)((c->V + 63) / 64);
    dirac_dd_split_kernel<<<blocks, 128, 0, st>>>(c->g, (const dd*)c->links_dd, (const dd*)c->clov_dd, in, out);
  }
  dw_note_launch();
}

// FP64 fields through double-float arithmetic: convert, apply, convert back (nrhs fields)
static int dirac_full_f64x(dw_ctx* c, const double* in, double* out, int nrhs, cudaStream_t st) {
  int rc = dw_make_dd(c, st);
  if (rc) return rc;
  const size_t n = (size_t)c->V * 24;
  dd *a = nullptr, *b = nullptr;
  DW_CUDA(cudaMallocAsync(&a, n * sizeof(dd), st));
  DW_CUDA(cudaMallocAsync(&b, n * sizeof(dd), st));
  for (int r = 0; r < nrhs; ++r) {
    f64_to_dd(in + r * n, a, n, st);
    dirac_full_dd(c, a, b, st);
    dd_to_f64(b, out + r * n, n, 0, st);
  }
  DW_CUDA(cudaFreeAsync(a, st));
  DW_CUDA(cudaFreeAsync(b, st));
  return DW_OK;
}

// bhat_e = eta_e - D_eo A_oo^{-1} eta_o, bhat_o = 0 (t: scratch field)
template <typename T>
void eo_prepare(dw_ctx* c, const T* eta, T* bhat, T* t, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  unsigned blocks = (unsigned)((c->V / 2 + 127) / 128);
  clover_inv_odd_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->clovinv[P], eta, t); dw_note_launch();
  eo_rhs_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], eta, t, bhat); dw_note_launch();
}
// psi_e = x_e, psi_o = A_oo^{-1}(eta_o - D_oe x_e)
template <typename T>
void eo_reconstruct(dw_ctx* c, const T* eta, const T* x, T* psi, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  unsigned blocks = (unsigned)((c->V / 2 + 127) / 128);
  eo_reconstruct_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clovinv[P], eta, x,
                                                   psi); dw_note_launch();
}
template void eo_prepare<double>(dw_ctx*, const double*, double*, double*, cudaStream_t);
template void eo_reconstruct<double>(dw_ctx*, const double*, const double*, double*, cudaStream_t);

template <typename T>
int dirac_schur(dw_ctx* c, const T* in, T* out, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  if (!c->sap_d[P]) DW_CUDA(cudaMalloc(&c->sap_d[P], dw_field_bytes(c, P)));
  T* t = (T*)c->sap_d[P];
  unsigned blocks = (unsigned)((c->V / 2 + 127) / 128);
  schur_odd_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clovinv[P], in, t); dw_note_launch();
  schur_even_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clov[P], in, t, out); dw_note_launch();
  return DW_OK;
}
template int dirac_schur<float>(dw_ctx*, const float*, float*, cudaStream_t);
template int dirac_schur<double>(dw_ctx*, const double*, double*, cudaStream_t);

extern "C" int dw_apply(dw_ctx* c, int prec, int op, int nrhs, const void* in, void* out, void* stream) {
  if (!c || !in || !out || in == out || nrhs < 1 || (prec != DW_F64 && prec != DW_F32 && prec != DW_F64X) ||
      (op != DW_OP_FULL && op != DW_OP_SCHUR) || (prec == DW_F64X && op != DW_OP_FULL)) {
    dw_set_error("dw_apply: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "dw_apply")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DW_F64X) {
    int rc = dirac_full_f64x(c, (const double*)in, (double*)out, nrhs, st);
    if (rc) return rc;
    DW_CUDA(cudaGetLastError());
    return DW_OK;
  }
  size_t n = (size_t)c->V * 24;
  if (nrhs > 1 && op == DW_OP_FULL) {   // multi-RHS kernel: links and clover read once per site
    if (prec == DW_F64) dirac_mrhs(c, (const double*)in, (double*)out, nrhs, c->tune_rgroup, st);
    else dirac_mrhs(c, (const float*)in, (float*)out, nrhs, c->tune_rgroup, st);
    DW_CUDA(cudaGetLastError());
    return DW_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    int rc = DW_OK;
    if (prec == DW_F64) {
      const double* a = (const double*)in + r * n;
      double* b = (double*)out + r * n;
      if (op == DW_OP_FULL) dirac_full(c, a, b, st); else rc = dirac_schur(c, a, b, st);
    } else {
      const float* a = (const float*)in + r * n;
      float* b = (float*)out + r * n;
      if (op == DW_OP_FULL) dirac_full(c, a, b, st); else rc = dirac_schur(c, a, b, st);
    }
    if (rc) return rc;
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

// ------------------------------------------------------------------ allocation-free Schur operator
// The even-odd Schur complement of dw_apply(DW_OP_SCHUR) with its odd-site intermediate
// A_oo^{-1} D_oe held in a fixed device array of this file instead of memory that the
// library allocates on first use.  For callers that must not allocate device memory at
// the time of the call: cudaMalloc synchronises the device (stalling work queued on other
// streams) and can fail in processes that run with a fixed memory reservation.
//
// The array holds one packed field, so the entry point serves volumes whose packed field
// fits in kSchurStaticBytes; larger ones are rejected with DW_EINVAL.  Every entry of the
// intermediate that is read is written earlier in the same call, so nothing has to start
// at zero.  All calls on one device share the array: calls that overlap in time (issued on
// different streams, or from several host threads without ordering) race on it.
namespace {
constexpr size_t kSchurStaticBytes = size_t(16) << 20;   // 16 MiB: FP64 up to 87381 sites, FP32 up to 174762
constexpr int kMaxDevices = 64;
std::mutex g_schur_static_mu;
void* g_schur_static_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_schur_static[kSchurStaticBytes];

// Address of the array on the current device, looked up once per device (the first call on a
// device does this set-up; make it before any stream capture).
static int schur_static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dw_cuda_fail(e, "dw_apply_schur_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    dw_set_error("dw_apply_schur_static: device ordinal beyond the supported range");
    return DW_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_schur_static_mu);
  if (!g_schur_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_schur_static);
    if (e != cudaSuccess) return dw_cuda_fail(e, "dw_apply_schur_static: cudaGetSymbolAddress");
    g_schur_static_ptr[dev] = p;
  }
  *out = g_schur_static_ptr[dev];
  return DW_OK;
}

template <typename T>
static void schur_static_launch(dw_ctx* c, const T* in, T* out, T* t, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  unsigned blocks = (unsigned)((c->V / 2 + 127) / 128);
  schur_odd_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clovinv[P], in, t); dw_note_launch();
  schur_even_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clov[P], in, t, out); dw_note_launch();
}

extern "C" int dw_apply_schur_static(dw_ctx* c, int prec, const void* in, void* out, void* stream) {
  if (!c || !in || !out || in == out || (prec != DW_F64 && prec != DW_F32)) {
    dw_set_error("dw_apply_schur_static: bad argument");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "dw_apply_schur_static")) return rc;
  const size_t need = dw_field_bytes(c, prec);
  if (need > kSchurStaticBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "dw_apply_schur_static: the intermediate field needs %zu bytes, more than the fixed %zu-byte "
             "device array (use dw_apply with DW_OP_SCHUR for this volume and precision)",
             need, kSchurStaticBytes);
    dw_set_error(msg);
    return DW_EINVAL;
  }
  void* t = nullptr;
  int rc = schur_static_scratch(&t);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DW_F64) schur_static_launch(c, (const double*)in, (double*)out, (double*)t, st);
  else schur_static_launch(c, (const float*)in, (float*)out, (float*)t, st);
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
