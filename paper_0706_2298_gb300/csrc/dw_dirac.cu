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

void dirac_full_dd(dw_ctx* c, const dd* in, dd* out, cudaStream_t st) {
  unsigned blocks = (unsigned)((c->V + 127) / 128);
  dirac_full_kernel<dd><<<blocks, 128, 0, st>>>(c->g, (const dd*)c->links_dd, (const dd*)c->clov_dd, in, out);
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

template <typename T>
static int dirac_schur(dw_ctx* c, const T* in, T* out, cudaStream_t st) {
  constexpr int P = prec_of<T>();
  if (!c->sap_d[P]) DW_CUDA(cudaMalloc(&c->sap_d[P], dw_field_bytes(c, P)));
  T* t = (T*)c->sap_d[P];
  unsigned blocks = (unsigned)((c->V / 2 + 127) / 128);
  schur_odd_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clovinv[P], in, t); dw_note_launch();
  schur_even_kernel<T><<<blocks, 128, 0, st>>>(c->g, (const T*)c->links[P], (const T*)c->clov[P], in, t, out); dw_note_launch();
  return DW_OK;
}

extern "C" int dw_apply(dw_ctx* c, int prec, int op, int nrhs, const void* in, void* out, void* stream) {
  if (!c || !in || !out || in == out || nrhs < 1 || (prec != DW_F64 && prec != DW_F32 && prec != DW_F64X) ||
      (op != DW_OP_FULL && op != DW_OP_SCHUR) || (prec == DW_F64X && op != DW_OP_FULL)) {
    dw_set_error("dw_apply: bad argument");
    return DW_EINVAL;
  }
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
