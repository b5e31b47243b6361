// Vector kernels on packed fields (flat arrays of complex numbers).
// Reductions accumulate in FP64 with a fixed order: per-thread partial
// sums, warp shuffles, one partial per CTA, and the last CTA to finish adds
// the CTA partials in index order -> results are deterministic.
#include "dw_common.cuh"

namespace {

constexpr int RB = 256;            // reduction CTA size
constexpr int RGRID = 608;         // 4 CTAs per SM on 152 SMs
constexpr int MAXK = 16;           // vectors per multi-dot launch

template <typename T, int K>
struct Ptrs {
  const T* p[K];
};

DW_D double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce NV doubles per thread over the grid into out[0..NV).  partial: RGRID*NV scratch.
template <int NV>
__device__ void grid_reduce(double* v, double* partial, unsigned* count, double* out) {
  __shared__ double sh[RB / 32][NV];
  __shared__ bool last;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[w][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0;
    for (int j = 0; j < RB / 32; ++j) s += sh[j][threadIdx.x];
    partial[blockIdx.x * NV + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(count, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA adds the CTA partials: warp w owns values k = w, w + 8, ...; lane q adds
  // partials q, q + 32, ... (independent loads, all in flight), then a fixed butterfly
  for (int k = w; k < NV; k += RB / 32) {
    double s = 0;
#pragma unroll 8
    for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(partial + b * NV + k);
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  if (threadIdx.x == 0) *count = 0;
}

// Per-thread partial sums in the field's own precision (FP32 fields: FP32, a few dozen terms per
// thread), combined across threads in FP64.  vec: 16-byte loads when both pointers allow them.
template <typename T>
__global__ void __launch_bounds__(RB) dot_kernel(const T* __restrict__ a, const T* __restrict__ b, size_t n,
                                                 int vec, double* partial, unsigned* count, double* out,
                                                 size_t sys_stride = 0) {
  // blockIdx.y: field of a batch (sys_stride reals apart), with its own scratch, counter and result
  a += blockIdx.y * sys_stride;
  b += blockIdx.y * sys_stride;
  partial += (size_t)blockIdx.y * gridDim.x * 3;
  count += blockIdx.y;
  out += 3 * blockIdx.y;
  T r0 = 0, r1 = 0, r2 = 0;   // re, im of (a, b), |a|^2
  const size_t tid = blockIdx.x * (size_t)RB + threadIdx.x, nth = (size_t)gridDim.x * RB;
  const cplx<T>* A = reinterpret_cast<const cplx<T>*>(a);
  const cplx<T>* B = reinterpret_cast<const cplx<T>*>(b);
  size_t done = 0;
  if (vec) {
    using U = typename Unit<T>::t;
    constexpr int C = Unit<T>::C;
    const U* AU = reinterpret_cast<const U*>(a);
    const U* BU = reinterpret_cast<const U*>(b);
    const size_t nu = n / C;
    for (size_t i = tid; i < nu; i += nth) {
      cplx<T> x[C], y[C];
      unpack_unit(AU[i], x);
      unpack_unit(BU[i], y);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        r0 += x[c].re * y[c].re + x[c].im * y[c].im;
        r1 += x[c].re * y[c].im - x[c].im * y[c].re;
        r2 += x[c].re * x[c].re + x[c].im * x[c].im;
      }
    }
    done = nu * C;
  }
  for (size_t i = done + tid; i < n; i += nth) {
    cplx<T> x = A[i], y = B[i];
    r0 += x.re * y.re + x.im * y.im;
    r1 += x.re * y.im - x.im * y.re;
    r2 += x.re * x.re + x.im * x.im;
  }
  double v[3] = {(double)r0, (double)r1, (double)r2};
  grid_reduce<3>(v, partial, count, out);
}

template <typename T, int K>
__global__ void __launch_bounds__(RB) multi_dot_kernel(Ptrs<T, MAXK> vs, const T* __restrict__ b, size_t n,
                                                       double* partial, unsigned* count, double* out,
                                                       size_t sys_stride = 0, size_t out_stride = 0) {
  // blockIdx.y: field of a batch (every vector and b sys_stride reals further on), own scratch
  const size_t so = blockIdx.y * sys_stride;
#pragma unroll
  for (int k = 0; k < K; ++k) vs.p[k] += so;
  b += so;
  partial += (size_t)blockIdx.y * gridDim.x * 2 * K;
  count += blockIdx.y;
  out += blockIdx.y * out_stride;
  T r[2 * K];
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) r[k] = 0;
  const cplx<T>* B = reinterpret_cast<const cplx<T>*>(b);
  for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
    cplx<T> y = B[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      cplx<T> x = reinterpret_cast<const cplx<T>*>(vs.p[k])[i];
      r[2 * k] += x.re * y.re + x.im * y.im;
      r[2 * k + 1] += x.re * y.im - x.im * y.re;
    }
  }
  double v[2 * K];
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) v[k] = (double)r[k];
  grid_reduce<2 * K>(v, partial, count, out);
}

// One GCR step for a batch of fields (grid.y = field r, fields sys_stride reals apart): chi_r *=
// inv_r, rho_r -= a_r chi_r, and |rho_r|^2 reduced as in dot_kernel (FP64 across threads); fields
// whose live flag is 0 are left alone.
struct GcrStepCoefs {
  float inv[16], ar[16], ai[16];
  int live[16];
};
template <typename T>
__global__ void __launch_bounds__(RB) gcr_step_batch_kernel(T* __restrict__ chi, T* __restrict__ rho, size_t n,
                                                            size_t sys_stride, GcrStepCoefs cf, double* partial,
                                                            unsigned* count, double* out) {
  const int r = blockIdx.y;
  if (!cf.live[r]) return;
  cplx<T>* X = reinterpret_cast<cplx<T>*>(chi + r * sys_stride);
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(rho + r * sys_stride);
  const T inv = cf.inv[r];
  const cplx<T> a = {(T)cf.ar[r], (T)cf.ai[r]};
  T nr = 0;
  for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
    const cplx<T> x = inv * X[i];
    X[i] = x;
    const cplx<T> y = Y[i] - a * x;
    Y[i] = y;
    nr += y.re * y.re + y.im * y.im;
  }
  double v[3] = {0.0, 0.0, (double)nr};
  grid_reduce<3>(v, partial + (size_t)r * gridDim.x * 3, count + r, out + 3 * r);
}

template <typename T>
__global__ void axpy_kernel(const T* __restrict__ x, T* __restrict__ y, T ar, T ai, size_t n) {
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(y);
  const cplx<T>* X = reinterpret_cast<const cplx<T>*>(x);
  cplx<T> a = {ar, ai};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Y[i] += a * X[i];
}
template <typename T>
__global__ void xpby_kernel(const T* __restrict__ x, T* __restrict__ y, T br, T bi, size_t n) {
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(y);
  const cplx<T>* X = reinterpret_cast<const cplx<T>*>(x);
  cplx<T> b = {br, bi};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Y[i] = X[i] + b * Y[i];
}
template <typename T>
__global__ void scale_kernel(T* __restrict__ x, T ar, T ai, size_t n) {
  cplx<T>* X = reinterpret_cast<cplx<T>*>(x);
  cplx<T> a = {ar, ai};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    X[i] = a * X[i];
}
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, double s, size_t n2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Tout)((double)x[i] * s);
}
// packed-field precision change: the unit layout differs between FP32 (2 complex per
// 16-byte unit) and FP64 (1 complex per unit), so convert site by site
template <typename Tin, typename Tout>
__global__ void field_convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, double s, size_t V) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    cplx<Tin> a[12];
    cplx<Tout> b[12];
    load_site<Tin, 12>(x, V, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = {(Tout)((double)a[k].re * s), (Tout)((double)a[k].im * s)};
    store_site<Tout, 12>(y, V, i, b);
  }
}
template <typename T>
struct Coefs {
  double c[2 * MAXK];
};
template <typename T, int K>
__global__ void multi_axpy_kernel(Ptrs<T, MAXK> vs, Coefs<T> cf, T* __restrict__ y, size_t n, int mode) {
  // mode 0: y -= sum c_k v_k ; mode 1: y = sum c_k v_k
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(y);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cplx<T> acc = mode == 0 ? Y[i] : cplx<T>{T(0), T(0)};
#pragma unroll
    for (int k = 0; k < K; ++k) {
      cplx<T> ck = {(T)cf.c[2 * k], (T)cf.c[2 * k + 1]};
      cplx<T> x = reinterpret_cast<const cplx<T>*>(vs.p[k])[i];
      if (mode == 0) acc -= ck * x; else acc += ck * x;
    }
    Y[i] = acc;
  }
}

// y_r -= sum_k c_{r,k} v_{k,r} for a batch of fields (grid.y = r; v_{k,r} = vs.p[k] + r sys_stride)
struct CoefsBatch {
  float c[16][2 * MAXK];
};
template <typename T, int K>
__global__ void multi_axpy_batch_kernel(Ptrs<T, MAXK> vs, CoefsBatch cf, T* __restrict__ y0, size_t n,
                                        size_t sys_stride) {
  const int rr = blockIdx.y;
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(y0 + rr * sys_stride);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cplx<T> acc = Y[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const cplx<T> ck = {(T)cf.c[rr][2 * k], (T)cf.c[rr][2 * k + 1]};
      acc -= ck * reinterpret_cast<const cplx<T>*>(vs.p[k] + rr * sys_stride)[i];
    }
    Y[i] = acc;
  }
}

inline unsigned ew_grid(size_t n) {
  size_t b = (n + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

template <typename T>
int blas_dot(dw_ctx* c, const T* a, const T* b, size_t n, double* out3, cudaStream_t s) {
  // out3 (device): re, im of (a, b) and |a|^2
  const int vec = ((((uintptr_t)a) | ((uintptr_t)b)) % 16) == 0;
  dot_kernel<T><<<RGRID, RB, 0, s>>>(a, b, n, vec, c->d_red, c->d_count, out3); dw_note_launch();
  return DW_OK;
}

// nrhs dot products (fields sys_stride reals apart) in one launch: out3[3 r ..] as blas_dot.
// At most 16 fields (their reduction counters); more are done one by one.
template <typename T>
int blas_dot_batch(dw_ctx* c, const T* a, const T* b, size_t n, size_t sys_stride, int nrhs, double* out3,
                   cudaStream_t s) {
  if (nrhs > 16) {
    for (int r = 0; r < nrhs; ++r) blas_dot<T>(c, a + r * sys_stride, b + r * sys_stride, n, out3 + 3 * r, s);
    return DW_OK;
  }
  const int vec = ((((uintptr_t)a) | ((uintptr_t)b) | (sys_stride * sizeof(T))) % 16) == 0;
  dot_kernel<T><<<dim3(RGRID / 4, nrhs), RB, 0, s>>>(a, b, n, vec, c->d_red, c->d_count + 16, out3, sys_stride);
  dw_note_launch();
  return DW_OK;
}
template int blas_dot_batch<float>(dw_ctx*, const float*, const float*, size_t, size_t, int, double*, cudaStream_t);
template int blas_dot_batch<double>(dw_ctx*, const double*, const double*, size_t, size_t, int, double*,
                                    cudaStream_t);

// chi_r *= inv_r, rho_r -= (ar_r + i ai_r) chi_r and |rho_r|^2 -> out3[3 r + 2] for the live fields
// of a batch of at most 16 (fields sys_stride reals apart), one launch.
int gcr_step_batch(dw_ctx* c, float* chi, float* rho, size_t n, size_t sys_stride, int nrhs, const double* inv,
                   const double* ar, const double* ai, const int* live, double* out3, cudaStream_t s) {
  if (nrhs > 16) return DW_EINVAL;
  GcrStepCoefs cf{};
  for (int r = 0; r < nrhs; ++r) {
    cf.inv[r] = (float)inv[r];
    cf.ar[r] = (float)ar[r];
    cf.ai[r] = (float)ai[r];
    cf.live[r] = live[r];
  }
  gcr_step_batch_kernel<float><<<dim3(RGRID / 4, nrhs), RB, 0, s>>>(chi, rho, n, sys_stride, cf, c->d_red,
                                                                    c->d_count + 16, out3);
  dw_note_launch();
  return DW_OK;
}

template <typename T, int K>
static void launch_md(dw_ctx* c, const Ptrs<T, MAXK>& p, const T* b, size_t n, double* out, cudaStream_t s) {
  multi_dot_kernel<T, K><<<RGRID, RB, 0, s>>>(p, b, n, c->d_red, c->d_count, out); dw_note_launch();
}

template <typename T>
int blas_multi_dot(dw_ctx* c, const T* const* vs, int k, const T* b, size_t n, double* out2, cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += MAXK) {
    int kk = k - j0 < MAXK ? k - j0 : MAXK;
    Ptrs<T, MAXK> p{};
    for (int j = 0; j < kk; ++j) p.p[j] = vs[j0 + j];
    double* o = out2 + 2 * j0;
    switch (kk) {
#define MD(K) case K: launch_md<T, K>(c, p, b, n, o, s); break;
      MD(1) MD(2) MD(3) MD(4) MD(5) MD(6) MD(7) MD(8) MD(9) MD(10) MD(11) MD(12) MD(13) MD(14) MD(15) MD(16)
#undef MD
    }
  }
  return DW_OK;
}

// The Gram-Schmidt pair of a batched GCR step for nrhs <= 16 fields (sys_stride reals apart):
// out[r ostride + 2j ..] = (v_j, b) for j < k, then (separately, with the coefficients the host
// formed) b -= sum_j c_{r,j} v_j.  One launch per chunk of 16 vectors instead of one per field.
template <typename T, int K>
static void launch_md_batch(dw_ctx* c, const Ptrs<T, MAXK>& p, const T* b, size_t n, size_t st, int nrhs,
                            double* out, size_t ostride, cudaStream_t s) {
  multi_dot_kernel<T, K><<<dim3(RGRID / 4, nrhs), RB, 0, s>>>(p, b, n, c->d_red, c->d_count + 16, out, st, ostride);
  dw_note_launch();
}
template <typename T>
int blas_multi_dot_batch(dw_ctx* c, const T* const* vs, int k, const T* b, size_t n, size_t sys_stride, int nrhs,
                         double* out, size_t ostride, cudaStream_t s) {
  if (nrhs > 16) return DW_EINVAL;
  for (int j0 = 0; j0 < k; j0 += MAXK) {
    const int kk = k - j0 < MAXK ? k - j0 : MAXK;
    Ptrs<T, MAXK> p{};
    for (int j = 0; j < kk; ++j) p.p[j] = vs[j0 + j];
    double* o = out + 2 * j0;
    switch (kk) {
#define MDB(K) case K: launch_md_batch<T, K>(c, p, b, n, sys_stride, nrhs, o, ostride, s); break;
      MDB(1) MDB(2) MDB(3) MDB(4) MDB(5) MDB(6) MDB(7) MDB(8) MDB(9) MDB(10) MDB(11) MDB(12) MDB(13) MDB(14)
      MDB(15) MDB(16)
#undef MDB
    }
  }
  return DW_OK;
}
template <typename T>
int blas_multi_axpy_batch(const T* const* vs, int k, const double* coef, size_t cstride, T* y, size_t n,
                          size_t sys_stride, int nrhs, cudaStream_t s) {
  if (nrhs > 16) return DW_EINVAL;
  for (int j0 = 0; j0 < k; j0 += MAXK) {
    const int kk = k - j0 < MAXK ? k - j0 : MAXK;
    Ptrs<T, MAXK> p{};
    CoefsBatch cf{};
    for (int j = 0; j < kk; ++j) p.p[j] = vs[j0 + j];
    for (int r = 0; r < nrhs; ++r)
      for (int j = 0; j < 2 * kk; ++j) cf.c[r][j] = (float)coef[r * cstride + 2 * j0 + j];
    const dim3 grid((ew_grid(n) + nrhs - 1) / nrhs + 1, nrhs);
    switch (kk) {
#define MAB(K) case K: multi_axpy_batch_kernel<T, K><<<grid, 256, 0, s>>>(p, cf, y, n, sys_stride); break;
      MAB(1) MAB(2) MAB(3) MAB(4) MAB(5) MAB(6) MAB(7) MAB(8) MAB(9) MAB(10) MAB(11) MAB(12) MAB(13) MAB(14)
      MAB(15) MAB(16)
#undef MAB
    }
    dw_note_launch();
  }
  return DW_OK;
}
template int blas_multi_dot_batch<float>(dw_ctx*, const float* const*, int, const float*, size_t, size_t, int,
                                         double*, size_t, cudaStream_t);
template int blas_multi_axpy_batch<float>(const float* const*, int, const double*, size_t, float*, size_t, size_t,
                                          int, cudaStream_t);

template <typename T>
void blas_axpy(const T* x, T* y, double ar, double ai, size_t n, cudaStream_t s) {
  axpy_kernel<T><<<ew_grid(n), 256, 0, s>>>(x, y, (T)ar, (T)ai, n); dw_note_launch();
}
template <typename T>
void blas_xpby(const T* x, T* y, double br, double bi, size_t n, cudaStream_t s) {
  xpby_kernel<T><<<ew_grid(n), 256, 0, s>>>(x, y, (T)br, (T)bi, n); dw_note_launch();
}
template <typename T>
void blas_scale(T* x, double ar, double ai, size_t n, cudaStream_t s) {
  scale_kernel<T><<<ew_grid(n), 256, 0, s>>>(x, (T)ar, (T)ai, n); dw_note_launch();
}
template <typename Tin, typename Tout>
void blas_convert(const Tin* x, Tout* y, double scale, size_t n, cudaStream_t s) {
  convert_kernel<Tin, Tout><<<ew_grid(2 * n), 256, 0, s>>>(x, y, scale, 2 * n); dw_note_launch();
}

template <typename Tin, typename Tout>
void field_convert(const Tin* x, Tout* y, double scale, size_t V, cudaStream_t s) {
  field_convert_kernel<Tin, Tout><<<ew_grid(V), 256, 0, s>>>(x, y, scale, V); dw_note_launch();
}

template <typename T, int K>
static void launch_ma(const Ptrs<T, MAXK>& p, const Coefs<T>& cf, T* y, size_t n, int mode, cudaStream_t s) {
  multi_axpy_kernel<T, K><<<ew_grid(n), 256, 0, s>>>(p, cf, y, n, mode); dw_note_launch();
}
template <typename T>
static void multi_axpy_impl(const T* const* vs, int k, const double* coef, T* y, size_t n, int mode,
                            cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += MAXK) {
    int kk = k - j0 < MAXK ? k - j0 : MAXK;
    Ptrs<T, MAXK> p{};
    Coefs<T> cf{};
    for (int j = 0; j < kk; ++j) {
      p.p[j] = vs[j0 + j];
      cf.c[2 * j] = coef[2 * (j0 + j)];
      cf.c[2 * j + 1] = coef[2 * (j0 + j) + 1];
    }
    int m = (j0 == 0) ? mode : 0;
    if (m == 1) {
      // first chunk of a linear combination: y = sum; later chunks: y += sum (negated coefs, mode 0)
    } else if (j0 > 0 && mode == 1) {
      for (int j = 0; j < 2 * kk; ++j) cf.c[j] = -cf.c[j];
    }
    switch (kk) {
#define MA(K) case K: launch_ma<T, K>(p, cf, y, n, m, s); break;
      MA(1) MA(2) MA(3) MA(4) MA(5) MA(6) MA(7) MA(8) MA(9) MA(10) MA(11) MA(12) MA(13) MA(14) MA(15) MA(16)
#undef MA
    }
  }
}
template <typename T>
void blas_multi_axpy(const T* const* vs, int k, const double* coef, T* y, size_t n, cudaStream_t s) {
  multi_axpy_impl(vs, k, coef, y, n, 0, s);
}
template <typename T>
void blas_lincomb(const T* const* vs, int k, const double* coef, T* out, size_t n, cudaStream_t s) {
  multi_axpy_impl(vs, k, coef, out, n, 1, s);
}

#define INST(T)                                                                                      \
  template int blas_dot<T>(dw_ctx*, const T*, const T*, size_t, double*, cudaStream_t);              \
  template int blas_multi_dot<T>(dw_ctx*, const T* const*, int, const T*, size_t, double*, cudaStream_t); \
  template void blas_axpy<T>(const T*, T*, double, double, size_t, cudaStream_t);                    \
  template void blas_xpby<T>(const T*, T*, double, double, size_t, cudaStream_t);                    \
  template void blas_scale<T>(T*, double, double, size_t, cudaStream_t);                             \
  template void blas_multi_axpy<T>(const T* const*, int, const double*, T*, size_t, cudaStream_t);   \
  template void blas_lincomb<T>(const T* const*, int, const double*, T*, size_t, cudaStream_t);
INST(float)
INST(double)
template void blas_convert<double, float>(const double*, float*, double, size_t, cudaStream_t);
template void blas_convert<float, double>(const float*, double*, double, size_t, cudaStream_t);
template void blas_convert<double, double>(const double*, double*, double, size_t, cudaStream_t);
template void blas_convert<float, float>(const float*, float*, double, size_t, cudaStream_t);
template void field_convert<double, float>(const double*, float*, double, size_t, cudaStream_t);
template void field_convert<float, double>(const float*, double*, double, size_t, cudaStream_t);
template void field_convert<double, double>(const double*, double*, double, size_t, cudaStream_t);
template void field_convert<float, float>(const float*, float*, double, size_t, cudaStream_t);

// ---------------------------------------------------------------- double-float conversions
namespace {

// double -> (hi, lo): hi = x with its fraction cut to 23 bits, lo = the remaining 29 bits rounded
// to FP32 (relative error <= 2^-48).  Integer operations only; zero, tiny (|x| < 2^-74), huge,
// infinite and NaN values take a plain conversion.
DW_D dd split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 949 || e > 1150) {
    const float h = __double2float_rz(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  const float lo = __uint2float_rn((unsigned)(b & 0x1FFFFFFFull)) * __uint_as_float((unsigned)(e - 948) << 23);
  return {hi, sign ? -lo : lo};
}
// FP32 -> FP64 by moving exponent and fraction (exact); zero and subnormal/special values aside
DW_D double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)((unsigned long long)u << 32));
  if (e == 0 || e == 255) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(e + 896) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__global__ void f64_to_dd_kernel(const double2* __restrict__ x, float4* __restrict__ y, size_t n2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    const dd a = split_double(v.x), b = split_double(v.y);
    y[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
  }
}
__global__ void dd_to_f64_kernel(const float4* __restrict__ x, double2* y, size_t n2, int add) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    double2 o = make_double2(widen(v.x) + widen(v.y), widen(v.z) + widen(v.w));
    if (add) {
      const double2 t = y[i];
      o.x += t.x;
      o.y += t.y;
    }
    y[i] = o;
  }
}

}  // namespace

void f64_to_dd(const double* x, dd* y, size_t n_real, cudaStream_t s) {
  const size_t n2 = n_real / 2;
  f64_to_dd_kernel<<<RGRID * 2, 256, 0, s>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<float4*>(y), n2);
  dw_note_launch();
}
void dd_to_f64(const dd* x, double* y, size_t n_real, int add, cudaStream_t s) {
  const size_t n2 = n_real / 2;
  dd_to_f64_kernel<<<RGRID * 2, 256, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<double2*>(y), n2,
                                            add);
  dw_note_launch();
}

int dw_make_dd(dw_ctx* c, cudaStream_t s) {
  if (c->links_dd) return DW_OK;
  const size_t nl = (size_t)c->V * 4 * 12, nc = (size_t)c->V * 72;   // reals (FP64 layouts)
  DW_CUDA(cudaMalloc(&c->links_dd, nl * sizeof(dd)));
  DW_CUDA(cudaMalloc(&c->clov_dd, nc * sizeof(dd)));
  f64_to_dd((const double*)c->links[DW_F64], (dd*)c->links_dd, nl, s);
  f64_to_dd((const double*)c->clov[DW_F64], (dd*)c->clov_dd, nc, s);
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
