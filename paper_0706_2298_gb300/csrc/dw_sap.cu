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

template <typename T>
int sap_apply(dw_ctx* c, int ncy, int nmr, const T* rho, T* xi, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  size_t bytes = dw_field_bytes(c, P);
  if (!c->sap_r[P]) DW_CUDA(cudaMalloc(&c->sap_r[P], bytes));
  if (!c->sap_d[P]) DW_CUDA(cudaMalloc(&c->sap_d[P], bytes));
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
template int sap_apply<float>(dw_ctx*, int, int, const float*, float*, cudaStream_t);
template int sap_apply<double>(dw_ctx*, int, int, const double*, double*, cudaStream_t);

extern "C" int sap_precondition(dw_ctx* c, int prec, int ncy, int nmr, int nrhs, const void* rho, void* xi,
                                void* stream) {
  if (!c || !rho || !xi || rho == xi || nrhs < 1 || nmr < 0 || (prec != DW_F64 && prec != DW_F32)) {
    dw_set_error("sap_precondition: bad argument");
    return DW_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = (size_t)c->V * 24;
  for (int r = 0; r < nrhs; ++r) {
    int rc = prec == DW_F64 ? sap_apply(c, ncy, nmr, (const double*)rho + r * n, (double*)xi + r * n, st)
                            : sap_apply(c, ncy, nmr, (const float*)rho + r * n, (float*)xi + r * n, st);
    if (rc) return rc;
  }
  return DW_OK;
}
