// Internal definitions shared by the CUDA translation units of libdwsolve.
//
// Packed device layout ("block-major SoA")
// ----------------------------------------
// Sites are ordered by Schwarz block: internal index
//     i = b * svol + p * shv + h
// with b the SAP block (lexicographic block coordinates, x0 slowest), p the
// site parity, h the position of the site among the block's sites of that
// parity in local lexicographic order (h = local_lex / 2; the last block
// extent is even so every pair of consecutive local sites holds one site
// of each parity).  Block origins have even coordinates, so local parity
// equals global parity.  Every Schwarz block is one contiguous index range,
// which is what the on-chip block solver stages.
//
// Per-site data are stored as structure of arrays in 16-byte units:
//   quark field : 12 complex  (k = 3*spin + colour)  -> 12*8/16 units (FP32: 6 float4, FP64: 12 double2)
//   link        : rows 0 and 1 of U_mu(x) (6 complex), row 2 rebuilt as conj(row0 x row1)
//   clover      : per chiral 6x6 Hermitian block 18 complex slots
//                 (slots 0..2 = real diagonal pairs, 3..17 = upper triangle row-major)
// Unit u of site i lives at plane u: base[u * V + i], so a warp touching 32
// consecutive sites reads 512 contiguous bytes per unit.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dwsolve.h"

#define DW_HD __host__ __device__ __forceinline__
#define DW_D __device__ __forceinline__

// ---------------------------------------------------------------- complex
template <typename T>
struct cplx {
  T re, im;
};
template <typename T> DW_HD cplx<T> mk(T r, T i) { return cplx<T>{r, i}; }
template <typename T> DW_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> DW_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> DW_HD cplx<T> operator-(cplx<T> a) { return {-a.re, -a.im}; }
template <typename T> DW_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> DW_HD cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> DW_HD cplx<T>& operator+=(cplx<T>& a, cplx<T> b) { a.re += b.re; a.im += b.im; return a; }
template <typename T> DW_HD cplx<T>& operator-=(cplx<T>& a, cplx<T> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename T> DW_HD cplx<T> conjg(cplx<T> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename T> DW_HD cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename T> DW_HD cplx<T> ti(cplx<T> a) { return {-a.im, a.re}; }
template <typename T> DW_HD T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------- 16-byte units
template <typename T> struct Unit;
template <> struct Unit<float> { using t = float4; static constexpr int C = 2; };
template <> struct Unit<double> { using t = double2; static constexpr int C = 1; };

DW_D void unpack_unit(const float4& v, cplx<float>* c) { c[0] = {v.x, v.y}; c[1] = {v.z, v.w}; }
DW_D void unpack_unit(const double2& v, cplx<double>* c) { c[0] = {v.x, v.y}; }
DW_D float4 pack_unit(const cplx<float>* c) { return make_float4(c[0].re, c[0].im, c[1].re, c[1].im); }
DW_D double2 pack_unit(const cplx<double>* c) { return make_double2(c[0].re, c[0].im); }

// ---------------------------------------------------------------- double-float ("dd") arithmetic
// A real number held as an unevaluated sum hi + lo of two FP32 values (|lo| <= ulp(hi)/2),
// about 48 significant bits.  Sums use Knuth's TwoSum, products Dekker's exact product formed
// with one FMA; both run on the FP32 pipes, whose rate on this part is many times the FP64 rate.
// Used where FP64-class accuracy is needed on large fields (restart residuals, restriction,
// prolongation).  Memory form: the FP64 layout with every double replaced by (hi, lo) floats.
struct dd {
  float hi, lo;
  dd() = default;
  DW_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  DW_HD constexpr dd(float f) : hi(f), lo(0.f) {}
  DW_HD constexpr dd(int i) : hi((float)i), lo(0.f) {}
  DW_HD dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
DW_D dd dd_two_sum(float a, float b) {        // exact: a + b = s + e
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
DW_D dd dd_quick_two_sum(float a, float b) {  // exact when |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
DW_D dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  return dd_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
DW_D dd operator-(dd a) { return {-a.hi, -a.lo}; }
DW_D dd operator-(dd a, dd b) { return a + (-b); }
DW_D dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                 // exact error of the leading product
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return dd_quick_two_sum(p, e);
}
DW_D dd& operator+=(dd& a, dd b) { a = a + b; return a; }
DW_D dd& operator-=(dd& a, dd b) { a = a - b; return a; }
DW_D double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }
DW_D dd __shfl_xor_sync(unsigned mask, dd v, int lane) {
  return {__shfl_xor_sync(mask, v.hi, lane), __shfl_xor_sync(mask, v.lo, lane)};
}
template <> struct Unit<dd> { using t = float4; static constexpr int C = 1; };
DW_D void unpack_unit(const float4& v, cplx<dd>* c) { c[0] = {dd(v.x, v.y), dd(v.z, v.w)}; }
DW_D float4 pack_unit(const cplx<dd>* c) { return make_float4(c[0].re.hi, c[0].re.lo, c[0].im.hi, c[0].im.lo); }

// load NC complex numbers of site i from unit planes (read-only path)
template <typename T, int NC>
DW_D void load_site(const T* __restrict__ base, size_t V, size_t i, cplx<T>* out) {
  using U = typename Unit<T>::t;
  constexpr int CU = Unit<T>::C;
  const U* p = reinterpret_cast<const U*>(base);
#pragma unroll
  for (int u = 0; u < NC / CU; ++u) unpack_unit(__ldg(p + (size_t)u * V + i), out + u * CU);
}
// plain (coherent) load, for buffers written earlier in the same kernel
template <typename T, int NC>
DW_D void load_site_rw(const T* base, size_t V, size_t i, cplx<T>* out) {
  using U = typename Unit<T>::t;
  constexpr int CU = Unit<T>::C;
  const U* p = reinterpret_cast<const U*>(base);
#pragma unroll
  for (int u = 0; u < NC / CU; ++u) unpack_unit(p[(size_t)u * V + i], out + u * CU);
}
template <typename T, int NC>
DW_D void store_site(T* __restrict__ base, size_t V, size_t i, const cplx<T>* in) {
  using U = typename Unit<T>::t;
  constexpr int CU = Unit<T>::C;
  U* p = reinterpret_cast<U*>(base);
#pragma unroll
  for (int u = 0; u < NC / CU; ++u) p[(size_t)u * V + i] = pack_unit(in + u * CU);
}

// ---------------------------------------------------------------- geometry
// Neighbour table entry for (parity p, half index h, direction d = 2*mu + (0 forward, 1 backward)):
// bits 0..14 = half index of the neighbour inside its block, bit 15 = neighbour in another block.
struct Geom {
  int L[4];
  long long V;
  int sb[4];
  int svol, shv, lsvol, lshv;    // block volume, half volume and their log2
  int nsap;                      // number of Schwarz blocks
  int antiperiodic;
  const uint16_t* nbtab;         // [2][shv][8]
  const int* blk_nb;             // [nsap][8]  neighbouring block in direction d
  const int* blk_x0;             // [nsap]     time coordinate of the block origin
  const uchar4* loc;             // [2][shv]   local coordinates (l0, l1, l2, l3)
};

struct SiteRef {
  int b, p, h;
};
DW_D SiteRef decode(const Geom& g, long long i) {
  SiteRef s;
  s.b = (int)(i >> g.lsvol);
  int w = (int)(i & (g.svol - 1));
  s.p = w >> g.lshv;
  s.h = w & (g.shv - 1);
  return s;
}
DW_D long long site_index(const Geom& g, int b, int p, int h) {
  return ((long long)b << g.lsvol) + (p << g.lshv) + h;
}
// neighbour of site (b, p, h) in direction d; sets *cross if the hop leaves the block
DW_D long long neighbour(const Geom& g, const SiteRef& s, int d, bool* cross) {
  uint16_t e = __ldg(g.nbtab + ((s.p * g.shv + s.h) << 3) + d);
  bool c = (e >> 15) != 0;
  *cross = c;
  int nb = c ? __ldg(g.blk_nb + s.b * 8 + d) : s.b;
  return site_index(g, nb, 1 - s.p, e & 0x7fff);
}
DW_D long long neighbour_of(const Geom& g, long long i, int d) {
  bool c;
  return neighbour(g, decode(g, i), d, &c);
}
// antiperiodic sign of a time hop: forward from x0 = L0-1, backward from x0 = 0
DW_D bool time_wrap(const Geom& g, const SiteRef& s, int d) {
  if (!g.antiperiodic || d > 1) return false;
  uchar4 l = __ldg(g.loc + s.p * g.shv + s.h);
  int x0 = __ldg(g.blk_x0 + s.b) + l.x;
  return d == 0 ? (x0 == g.L[0] - 1) : (x0 == 0);
}

// ---------------------------------------------------------------- SU(3)
template <typename T>
struct SU3 {
  cplx<T> m[3][3];
};
template <typename T>
DW_D void load_link(const T* __restrict__ links, size_t V, int mu, size_t i, SU3<T>& U) {
  cplx<T> r[6];
  load_site<T, 6>(links + (size_t)mu * 12 * V, V, i, r);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    U.m[0][j] = r[j];
    U.m[1][j] = r[3 + j];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    U.m[2][j] = conjg(U.m[0][j1] * U.m[1][j2] - U.m[0][j2] * U.m[1][j1]);
  }
}
template <typename T>
DW_D void su3_mul(const SU3<T>& U, const cplx<T>* h, cplx<T>* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = U.m[a][0] * h[0] + U.m[a][1] * h[1] + U.m[a][2] * h[2];
}
template <typename T>
DW_D void su3_dag_mul(const SU3<T>& U, const cplx<T>* h, cplx<T>* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = cmulc(U.m[0][a], h[0]) + cmulc(U.m[1][a], h[1]) + cmulc(U.m[2][a], h[2]);
}

// ---------------------------------------------------------------- spin structure
// gamma_mu = [[0, e_mu], [e_mu^+, 0]] with e_0 = -1, e_k = -i sigma_k.
// (1 + S gamma_mu) psi = [h ; S e_mu^+ h],  h = psi_up + S e_mu psi_lo  (S = +-1).
template <int MU, typename T>
DW_D void e_mul(const cplx<T>& l2, const cplx<T>& l3, cplx<T>& v0, cplx<T>& v1) {
  if (MU == 0) { v0 = -l2; v1 = -l3; }
  if (MU == 1) { v0 = -ti(l3); v1 = -ti(l2); }
  if (MU == 2) { v0 = -l3; v1 = l2; }
  if (MU == 3) { v0 = -ti(l2); v1 = ti(l3); }
}
template <int MU, typename T>
DW_D void edag_mul(const cplx<T>& h0, const cplx<T>& h1, cplx<T>& w0, cplx<T>& w1) {
  if (MU == 0) { w0 = -h0; w1 = -h1; }
  if (MU == 1) { w0 = ti(h1); w1 = ti(h0); }
  if (MU == 2) { w0 = h1; w1 = -h0; }
  if (MU == 3) { w0 = ti(h0); w1 = -ti(h1); }
}

// acc += sign * (1 + S gamma_mu) W psi, W = U (DAG=false) or U^+ (DAG=true)
template <int MU, int S, bool DAG, typename T>
DW_D void hop_acc(cplx<T>* acc, const cplx<T>* psi, const SU3<T>& U, T sign) {
  cplx<T> h[2][3], w[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<T> v0, v1;
    e_mul<MU>(psi[6 + c], psi[9 + c], v0, v1);
    if (S > 0) { h[0][c] = psi[c] + v0; h[1][c] = psi[3 + c] + v1; }
    else       { h[0][c] = psi[c] - v0; h[1][c] = psi[3 + c] - v1; }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (DAG) su3_dag_mul(U, h[a], w[a]); else su3_mul(U, h[a], w[a]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<T> l0, l1;
    edag_mul<MU>(w[0][c], w[1][c], l0, l1);
    acc[c] += sign * w[0][c];
    acc[3 + c] += sign * w[1][c];
    if (S > 0) { acc[6 + c] += sign * l0; acc[9 + c] += sign * l1; }
    else       { acc[6 + c] -= sign * l0; acc[9 + c] -= sign * l1; }
  }
}

// ---------------------------------------------------------------- clover
// y = A x for one chiral block stored in 18 slots (see layout above)
template <typename T>
DW_D void herm6_mul(const cplx<T>* s, const cplx<T>* x, cplx<T>* y) {
  const T d[6] = {s[0].re, s[0].im, s[1].re, s[1].im, s[2].re, s[2].im};
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = d[i] * x[i];
  int k = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      y[i] += s[k] * x[j];
      y[j] += cmulc(s[k], x[i]);
      ++k;
    }
  }
}
template <typename T>
DW_D void clover_apply(const T* __restrict__ clov, size_t V, size_t i, const cplx<T>* x, cplx<T>* y) {
  cplx<T> s[18];
  load_site<T, 18>(clov, V, i, s);
  herm6_mul(s, x, y);
  load_site<T, 18>(clov + 36 * V, V, i, s);
  herm6_mul(s, x + 6, y + 6);
}

// ---------------------------------------------------------------- contexts
struct HostTimer;

// Device buffers kept by a context between calls: a solver asks for the same sequence of sizes
// on every call and gets the same buffers back (allocated on the first call, or when a larger
// size is asked for), so repeated solves allocate and free nothing.
struct WsArena {
  std::vector<std::pair<size_t, void*>> bufs;
  size_t next = 0;
  void rewind() { next = 0; }
  cudaError_t get(size_t bytes, void** p) {
    if (next < bufs.size() && bufs[next].first >= bytes) { *p = bufs[next++].second; return cudaSuccess; }
    if (next < bufs.size()) {        // too small: replace this buffer
      cudaFree(bufs[next].second);
      bufs[next] = {0, nullptr};
    } else {
      bufs.push_back({0, nullptr});
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    bufs[next++] = {bytes, *p};
    return cudaSuccess;
  }
  void release() {
    for (auto& b : bufs)
      if (b.second) cudaFree(b.second);
    bufs.clear();
    next = 0;
  }
};

struct dw_ctx {
  dw_params p;
  int device = -1;             // CUDA device the context's memory lives on (current device at dw_create)
  uint64_t gauge_hash = 0;     // FNV-1a hash of the links given to dw_create (identifies the gauge field)
  Geom g;                      // device pointers filled in
  long long V;
  int nsb[4];
  std::vector<int> canon_of;   // internal index -> canonical site (host copy)
  std::vector<int> blk_colour; // per Schwarz block
  int* d_canon_of = nullptr;
  uint16_t* d_nbtab = nullptr;
  int* d_blk_nb = nullptr;
  int* d_blk_x0 = nullptr;
  uchar4* d_loc = nullptr;
  int* d_colour_list = nullptr;  // blocks of colour 0 then colour 1
  int ncolour[2] = {0, 0};
  void* links[2] = {nullptr, nullptr};    // [DW_F64], [DW_F32]
  void* clov[2] = {nullptr, nullptr};
  void* clovinv[2] = {nullptr, nullptr};
  void* links_dd = nullptr;               // double-float copies (made on first use)
  void* clov_dd = nullptr;
  void* sap_r[2] = {nullptr, nullptr};    // SAP residual workspace
  void* sap_d[2] = {nullptr, nullptr};    // SAP last-correction workspace
  int sap_cap = 1;                        // right-hand sides the FP32 SAP workspace holds
  int tune_rgroup = 0;                    // multi-RHS D variant: 0 interleaved, 1..3 per pass (autotuned)
  int tune_sap_staged = 1;                // 1: staged FP32 Schwarz kernel, 0: generic kernel (autotuned)
  void* graph_cache = nullptr;            // captured M_sap launch sequences (dw_sap.cu)
  cudaStream_t cap_stream = nullptr;      // stream used only for graph capture
  double* d_red = nullptr;                // reduction scratch
  unsigned* d_count = nullptr;
  double* h_red = nullptr;                // pinned host mirror
  WsArena ws_solve[4];                    // solver workspaces: [0] GCR, [1] batched GCR, [2] CGNR and
                                          // BiCGstab, [3] low-mode subspace iteration
};

// DW_OK when the calling thread's current device is the context's device; otherwise DW_EINVAL
// with a message naming the entry point (kernels would mix memory of two devices).
int dw_check_device(const dw_ctx* c, const char* who);


// ---------------------------------------------------------------- mbarriers and bulk copies (sm_90+)
DW_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
DW_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
DW_D void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
DW_D void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
DW_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait for the completion of the phase with this parity: false (and the error flag set)
// if it has not completed after ~2^26 polls
DW_D bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long it = 0; it < (1LL << 26); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}
DW_D void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// kernel launch counter (process-wide, all devices) ---------------------------
void dw_note_launch();

// error handling ------------------------------------------------------------
void dw_set_error(const std::string& msg);
int dw_cuda_fail(cudaError_t e, const char* what);
#define DW_CUDA(call)                                      \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return dw_cuda_fail(_e, #call); \
  } while (0)

template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? DW_F64 : DW_F32; }
inline size_t real_size(int prec) { return prec == DW_F64 ? 8 : 4; }

// launch helpers implemented in dw_blas.cu -------------------------------------
// Reductions: per-thread partial sums in the field precision, combined in FP64 in a fixed order
// (deterministic).
template <typename T> int blas_dot(dw_ctx* c, const T* a, const T* b, size_t n_cplx, double* out2, cudaStream_t s);
template <typename T> int blas_multi_dot(dw_ctx* c, const T* const* vs, int k, const T* b, size_t n_cplx,
                                         double* out2, cudaStream_t s);
// nrhs dots of fields sys_stride reals apart in one launch (results 3 per field, as blas_dot)
template <typename T> int blas_dot_batch(dw_ctx* c, const T* a, const T* b, size_t n_cplx, size_t sys_stride,
                                         int nrhs, double* out3, cudaStream_t s);
// Gram-Schmidt of a batch (<= 16 fields, sys_stride reals apart): dots of k vectors with b, and
// b -= sum_j c_{r,j} v_j with host coefficients coef[r cstride + 2j ..]
template <typename T> int blas_multi_dot_batch(dw_ctx* c, const T* const* vs, int k, const T* b, size_t n_cplx,
                                               size_t sys_stride, int nrhs, double* out, size_t ostride,
                                               cudaStream_t s);
template <typename T> int blas_multi_axpy_batch(const T* const* vs, int k, const double* coef, size_t cstride, T* y,
                                                size_t n_cplx, size_t sys_stride, int nrhs, cudaStream_t s);
// one GCR step for live fields of a batch (<= 16): chi_r *= inv_r, rho_r -= a_r chi_r, |rho_r|^2
int gcr_step_batch(dw_ctx* c, float* chi, float* rho, size_t n_cplx, size_t sys_stride, int nrhs, const double* inv,
                   const double* ar, const double* ai, const int* live, double* out3, cudaStream_t s);
// y = a*x + y  (complex a)
template <typename T> void blas_axpy(const T* x, T* y, double ar, double ai, size_t n_cplx, cudaStream_t s);
// y = x + b*y  (complex b)
template <typename T> void blas_xpby(const T* x, T* y, double br, double bi, size_t n_cplx, cudaStream_t s);
template <typename T> void blas_scale(T* x, double ar, double ai, size_t n_cplx, cudaStream_t s);
// flat complex arrays (little vectors, matrices) only -- not packed fields of mixed precision
template <typename Tin, typename Tout> void blas_convert(const Tin* x, Tout* y, double scale, size_t n_cplx,
                                                        cudaStream_t s);
// packed fields of V sites: y = scale * x with a change of precision (layouts differ per precision)
template <typename Tin, typename Tout> void field_convert(const Tin* x, Tout* y, double scale, size_t V,
                                                         cudaStream_t s);
// y -= sum_j coef[j] * vs[j]  (coef: host array of k complex)
template <typename T> void blas_multi_axpy(const T* const* vs, int k, const double* coef, T* y, size_t n_cplx,
                                           cudaStream_t s);
// out = sum_j coef[j] * vs[j]
template <typename T> void blas_lincomb(const T* const* vs, int k, const double* coef, T* out, size_t n_cplx,
                                        cudaStream_t s);

// double-float fields (dd form: the FP64 layout with each double as (hi, lo) floats), n reals
void f64_to_dd(const double* x, dd* y, size_t n_real, cudaStream_t s);
// y = dd(x) (add = 0) or y += dd(x) (add = 1), in FP64
void dd_to_f64(const dd* x, double* y, size_t n_real, int add, cudaStream_t s);
// make the context's double-float copies of the links and the clover term (once)
int dw_make_dd(dw_ctx* c, cudaStream_t s);
// out = D in on dd-form fields (FP64-class accuracy on the FP32 pipes)
void dirac_full_dd(dw_ctx* c, const dd* in, dd* out, cudaStream_t s);

// dirac / sap entry points used by the solver ---------------------------------------
// even-odd Schur operator (odd sites of out zero; uses the context's scratch field) and the
// preparation / reconstruction of the even-odd system
template <typename T> int dirac_schur(dw_ctx* c, const T* in, T* out, cudaStream_t s);
template <typename T> void eo_prepare(dw_ctx* c, const T* eta, T* bhat, T* t, cudaStream_t s);
template <typename T> void eo_reconstruct(dw_ctx* c, const T* eta, const T* x, T* psi, cudaStream_t s);
template <typename T> void dirac_full(dw_ctx* c, const T* in, T* out, cudaStream_t s);
// nrhs fields stored consecutively; rgroup right-hand sides share one pass over the links
template <typename T> void dirac_mrhs(dw_ctx* c, const T* in, T* out, int nrhs, int rgroup, cudaStream_t s);
template <typename T> int sap_apply(dw_ctx* c, int ncy, int nmr, const T* rho, T* xi, cudaStream_t s);
int sap_apply_mrhs(dw_ctx* c, int ncy, int nmr, const float* rho, float* xi, int nrhs, cudaStream_t s);
// same, replayed from a captured CUDA graph after the first call for a (rho, xi, nrhs, ncy, nmr) key
int sap_apply_mrhs_graph(dw_ctx* c, int ncy, int nmr, const float* rho, float* xi, int nrhs, cudaStream_t s);
void sap_graphs_free(dw_ctx* c);

// ---------------------------------------------------------------- hopping term
// acc += sign * (1 - gamma_mu) U_mu(x) psi(x+mu) + sign * (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)
// for one direction mu (sign = -1 across the antiperiodic time boundary).
// The caller multiplies the sum by -1/2.
template <int MU, typename T>
DW_D void hop_dir(const Geom& g, const SiteRef& s, long long i, const T* __restrict__ links,
                  const T* __restrict__ in, cplx<T>* acc) {
  const size_t V = g.V;
  bool cr;
  SU3<T> U;
  cplx<T> p[12];
  long long j = neighbour(g, s, 2 * MU, &cr);
  T sg = time_wrap(g, s, 2 * MU) ? T(-1) : T(1);
  load_link(links, V, MU, i, U);
  load_site<T, 12>(in, V, j, p);
  hop_acc<MU, -1, false>(acc, p, U, sg);
  j = neighbour(g, s, 2 * MU + 1, &cr);
  sg = time_wrap(g, s, 2 * MU + 1) ? T(-1) : T(1);
  load_link(links, V, MU, j, U);
  load_site<T, 12>(in, V, j, p);
  hop_acc<MU, +1, true>(acc, p, U, sg);
}
template <typename T>
DW_D void hop_all(const Geom& g, const SiteRef& s, long long i, const T* __restrict__ links,
                  const T* __restrict__ in, cplx<T>* acc) {
  hop_dir<0>(g, s, i, links, in, acc);
  hop_dir<1>(g, s, i, links, in, acc);
  hop_dir<2>(g, s, i, links, in, acc);
  hop_dir<3>(g, s, i, links, in, acc);
}
