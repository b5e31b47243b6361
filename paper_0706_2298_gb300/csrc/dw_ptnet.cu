// Gauge-covariant parallel-transport network (learned subspace generation).
//
// A layer maps C_in channel fields h_c (each a quark field) to C_out fields:
//     h'_{c'}(x) = sum_{d=0..8} sum_c W_d[c' s', c s] (T_d h_c)(x)
// with T_0 = 1, T_{1+2mu} h(x) = U_mu(x) h(x+mu), T_{2+2mu} h(x) = U_mu(x-mu)^+ h(x-mu)
// (fermion links, antiperiodic sign across the time boundary).  W acts on (channel, spin), the
// transports on (site, colour), so the two commute and the adjoint layer
//     g_c(x) = sum_d sum_{c'} W_d^+ (T_d^+ g')(x)
// has the same form with W -> W^+ and T_{+mu} <-> T_{-mu}.  This is the data gradient used in
// back-propagation.  The weight gradient is dW_d = sum_{x, colour} g'(x) (T_d h)(x)^+.
//
// Weights: per layer 9 x (4 C_out) x (4 C_in) complex (FP32), layers stored back to back.
// Channel fields are packed FP32 fields stored one after the other.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "dw_common.cuh"

namespace {

constexpr int PT_THREADS = 128;

// transport of one channel field along PTNet direction d (0 = none) to site s/i; out[4][3]
DW_D void pt_transport(const Geom& g, const float* __restrict__ links, const float* __restrict__ f,
                       const SiteRef& s, long long i, int d, cplx<float> (*o)[3]) {
  const size_t V = g.V;
  cplx<float> p[12];
  if (d == 0) {
    load_site<float, 12>(f, V, i, p);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) o[sp][a] = p[3 * sp + a];
    return;
  }
  const int nd = d - 1, mu = nd >> 1;
  bool cr;
  const long long j = neighbour(g, s, nd, &cr);
  const float sg = time_wrap(g, s, nd) ? -1.f : 1.f;
  SU3<float> U;
  load_link(links, V, mu, (nd & 1) ? j : i, U);
  load_site<float, 12>(f, V, j, p);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    cplx<float> w[3];
    if (nd & 1) su3_dag_mul(U, p + 3 * sp, w); else su3_mul(U, p + 3 * sp, w);
#pragma unroll
    for (int a = 0; a < 3; ++a) o[sp][a] = sg * w[a];
  }
}

// one layer (ADJ = false) or its adjoint (ADJ = true); thread = (site, output channel)
template <int CIN, int COUT, bool ADJ>
__global__ void __launch_bounds__(PT_THREADS) ptnet_layer_kernel(Geom g, const float* __restrict__ links,
                                                                 const float2* __restrict__ W,
                                                                 const float* __restrict__ in,
                                                                 float* __restrict__ out) {
  constexpr int NI = ADJ ? COUT : CIN;      // channels read
  constexpr int NO = ADJ ? CIN : COUT;      // channels written
  constexpr int SPB = PT_THREADS / NO;      // sites per block
  __shared__ float2 sW[4 * NO][4 * NI];
  const int t = threadIdx.x;
  const int co = t % NO, sl = t / NO;
  const long long i = (long long)blockIdx.x * SPB + sl;
  const bool valid = sl < SPB && i < g.V;
  const size_t fs = (size_t)g.V * 24;
  SiteRef s = decode(g, valid ? i : 0);
  cplx<float> acc[4][3];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[sp][a] = {0.f, 0.f};
  for (int d = 0; d < 9; ++d) {
    __syncthreads();
    const float2* Wd = W + (size_t)d * (4 * COUT) * (4 * CIN);
    for (int e = t; e < 16 * NO * NI; e += PT_THREADS) {
      const int r = e / (4 * NI), c = e % (4 * NI);
      // forward: sW = W_d [4 COUT][4 CIN]; adjoint: sW = W_d^+ [4 CIN][4 COUT]
      float2 w = ADJ ? Wd[(size_t)c * (4 * CIN) + r] : Wd[(size_t)r * (4 * CIN) + c];
      sW[r][c] = ADJ ? make_float2(w.x, -w.y) : w;
    }
    __syncthreads();
    if (!valid) continue;
    // adjoint transport: T_{+mu}^+ has the form of T_{-mu} and vice versa
    const int dt = (ADJ && d > 0) ? (((d - 1) ^ 1) + 1) : d;
    for (int ci = 0; ci < NI; ++ci) {
      cplx<float> th[4][3];
      pt_transport(g, links, in + (size_t)ci * fs, s, i, dt, th);
#pragma unroll
      for (int so = 0; so < 4; ++so) {
#pragma unroll
        for (int si = 0; si < 4; ++si) {
          const float2 w = sW[4 * co + so][4 * ci + si];
          const cplx<float> wc = {w.x, w.y};
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[so][a] += wc * th[si][a];
        }
      }
    }
  }
  if (!valid) return;
  cplx<float> o[12];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) o[3 * sp + a] = acc[sp][a];
  store_site<float, 12>(out + (size_t)co * fs, g.V, i, o);
}

// partial weight gradients: CTA (chunk, d) sums g'(x) (T_d h)(x)^+ over its sites
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) ptnet_dw_kernel(Geom g, const float* __restrict__ links,
                                                       const float* __restrict__ gout,
                                                       const float* __restrict__ h, float2* partial,
                                                       long long chunk) {
  constexpr int S = 8;                         // sites per tile
  constexpr int E = 16 * COUT * CIN;           // entries of W_d
  constexpr int EPT = (E + 255) / 256;         // entries per thread
  __shared__ cplx<float> sg[S][4 * COUT][3];
  __shared__ cplx<float> sx[S][4 * CIN][3];
  const int d = blockIdx.y;
  const long long i0 = (long long)blockIdx.x * chunk, i1 = min(i0 + chunk, (long long)g.V);
  const size_t fs = (size_t)g.V * 24;
  // per entry: the sum of a tile (S sites x 3 colours, 24 products) is formed in FP32 and
  // folded into a compensated (Kahan) FP32 accumulator, so that the error of a chunk's sum does
  // not grow with the number of sites it covers
  cplx<float> acc[EPT], cmp[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) { acc[k] = {0.f, 0.f}; cmp[k] = {0.f, 0.f}; }
  for (long long b0 = i0; b0 < i1; b0 += S) {
    __syncthreads();
    for (int w = threadIdx.x; w < S * (COUT + CIN); w += 256) {
      const int sl = w % S, job = w / S;
      const long long i = b0 + sl;
      if (i >= i1) {
        if (job < COUT) { for (int r = 0; r < 4; ++r) for (int a = 0; a < 3; ++a) sg[sl][4 * job + r][a] = {0.f, 0.f}; }
        else { const int c = job - COUT; for (int r = 0; r < 4; ++r) for (int a = 0; a < 3; ++a) sx[sl][4 * c + r][a] = {0.f, 0.f}; }
        continue;
      }
      if (job < COUT) {
        cplx<float> p[12];
        load_site<float, 12>(gout + (size_t)job * fs, g.V, i, p);
        for (int r = 0; r < 4; ++r) for (int a = 0; a < 3; ++a) sg[sl][4 * job + r][a] = p[3 * r + a];
      } else {
        const int c = job - COUT;
        cplx<float> th[4][3];
        SiteRef s = decode(g, i);
        pt_transport(g, links, h + (size_t)c * fs, s, i, d, th);
        for (int r = 0; r < 4; ++r) for (int a = 0; a < 3; ++a) sx[sl][4 * c + r][a] = th[r][a];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < E) {
        const int r = e / (4 * CIN), c = e % (4 * CIN);
        cplx<float> tile = {0.f, 0.f};
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
          for (int a = 0; a < 3; ++a) tile += cmulc(sx[sl][c][a], sg[sl][r][a]);
        const float yr = tile.re - cmp[k].re, yi = tile.im - cmp[k].im;
        const float tr = acc[k].re + yr, tq = acc[k].im + yi;
        cmp[k] = {(tr - acc[k].re) - yr, (tq - acc[k].im) - yi};
        acc[k] = {tr, tq};
      }
    }
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + 256 * k;
    if (e < E) partial[((size_t)blockIdx.x * 9 + d) * E + e] = make_float2(acc[k].re, acc[k].im);
  }
}

// grad[d][e] = scale * sum over chunks (fixed order)
__global__ void ptnet_dw_reduce_kernel(const float2* __restrict__ partial, int nchunk, int E, float scale,
                                       float2* grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * E) return;
  double re = 0, im = 0;
  for (int c = 0; c < nchunk; ++c) {
    float2 v = partial[(size_t)c * 9 * E + t];
    re += v.x;
    im += v.y;
  }
  grad[t] = make_float2((float)(scale * re), (float)(scale * im));
}

// Adam on real and imaginary parts
__global__ void ptnet_adam_kernel(size_t n, float* w, const float* gr, float* m, float* v, float lr, float b1,
                                  float b2, float eps, float c1, float c2) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float g = gr[t];
  const float mt = b1 * m[t] + (1.f - b1) * g;
  const float vt = b2 * v[t] + (1.f - b2) * g * g;
  m[t] = mt;
  v[t] = vt;
  w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

template <int CIN, int COUT, bool ADJ>
void launch_layer(dw_ctx* c, const float2* W, const float* in, float* out, cudaStream_t st) {
  constexpr int NO = ADJ ? CIN : COUT;
  constexpr int SPB = PT_THREADS / NO;
  const unsigned blocks = (unsigned)((c->V + SPB - 1) / SPB);
  ptnet_layer_kernel<CIN, COUT, ADJ><<<blocks, PT_THREADS, 0, st>>>(c->g, (const float*)c->links[DW_F32], W, in,
                                                                    out); dw_note_launch();
}

// ------------------------------------------------------------------ tensor-core 16 -> 16 layer
// The 16-channel layer is a dense complex contraction per site and colour: out = sum_d W_d (T_d h)
// with W_d a 64 x 64 complex matrix on (channel, spin).  In real form it is one GEMM per CTA tile:
//   D[128 x 192] += A_d[128 x 128] B_d[128 x 192],  d = 0..8
// A_d = [[Re W_d, -Im W_d], [Im W_d, Re W_d]] (rows: output (channel, spin) x (re, im)), B_d the
// transported input of 64 sites x 3 colours (columns) by (channel, spin) x (re, im) (rows), BF16
// operands in shared memory, the FP32 accumulator in tensor memory (tcgen05.mma, kind::f16, one
// elected thread issues).  A_d is staged by a bulk copy from a pre-arranged image; B_d is built by
// all threads (parallel transport on the CUDA cores, rounded to BF16).  Two stages: the
// transports of direction d + 1 overlap the MMAs of direction d.  Operands are K-major without
// swizzle: 8 x 16-byte core matrices, K-adjacent ones 128 bytes apart (leading byte offset),
// 8-row groups 2048 bytes apart (stride byte offset).
constexpr int TC_M = 128, TC_K = 128;
constexpr int TC_THREADS = 256;
constexpr int TC_A_BYTES = TC_M * TC_K * 2;    // 32 KB
// per tile of S sites (S = 64: one CTA per SM; S = 32: two, for more warps hiding the transports)
template <int S>
struct TcTile {
  static constexpr int N = 3 * S;                              // columns: (site, colour)
  static constexpr int B_BYTES = N * TC_K * 2;                 // 48 KB / 24 KB
  static constexpr uint32_t TMEM_COLS = N <= 128 ? 128u : 256u;
  static constexpr int STAGE_LD = N + 1;                       // FP32 staging row stride (bank-conflict free)
  static constexpr size_t SMEM = 2 * TC_A_BYTES + 2 * B_BYTES + 128;   // two per SM fit at S = 32
  static constexpr int MIN_BLOCKS = S <= 32 ? 2 : 1;
  // instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N = 3S, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                    ((uint32_t)(TC_M >> 4) << 24);
};

// byte offset of element (row, k) in a K-major no-swizzle operand with K = 128
DW_HD uint32_t tc_off(int row, int k) {
  return (uint32_t)((row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
DW_D uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;             // leading byte offset: next core matrix along K
  d |= (uint64_t)(2048 >> 4) << 32;            // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                      // descriptor version of tcgen05; no swizzle
  return d;
}

DW_D void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum) : "memory");
}
DW_D void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
DW_D void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
DW_D void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
DW_D void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// A_d images of one 16 -> 16 layer (ADJ: of W_d^+), BF16 in the core-matrix layout
template <bool ADJ>
__global__ void ptnet_tc_pack_kernel(const float2* __restrict__ W, __nv_bfloat16* A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * TC_M * TC_K) return;
  const int d = t / (TC_M * TC_K), e = t % (TC_M * TC_K), r = e / TC_K, k = e % TC_K;
  const int ro = r & 63, ko = k & 63;
  const float2* Wd = W + (size_t)d * 64 * 64;
  float2 w = ADJ ? Wd[ko * 64 + ro] : Wd[ro * 64 + ko];
  if (ADJ) w.y = -w.y;
  const float val = r < 64 ? (k < 64 ? w.x : -w.y) : (k < 64 ? w.y : w.x);
  A[(size_t)d * TC_M * TC_K + tc_off(r, k) / 2] = __float2bfloat16_rn(val);
}

template <bool ADJ, int S>
__global__ void __launch_bounds__(TC_THREADS, TcTile<S>::MIN_BLOCKS) ptnet_tc_layer_kernel(Geom g, const float* __restrict__ links,
                                                                       const __nv_bfloat16* __restrict__ Apack,
                                                                       const float* __restrict__ in,
                                                                       float* __restrict__ out, int* err) {
  using TT = TcTile<S>;
  extern __shared__ uint8_t tc_raw[];
  __shared__ uint64_t bar_tma[2], bar_mma[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const uint32_t raw = smem_u32(tc_raw);
  uint8_t* sb = tc_raw + (((raw + 127u) & ~127u) - raw);         // 128-byte aligned operand area
  uint8_t* abuf[2] = {sb, sb + TC_A_BYTES};
  uint8_t* bbuf[2] = {sb + 2 * TC_A_BYTES, sb + 2 * TC_A_BYTES + TT::B_BYTES};
  float* stage = reinterpret_cast<float*>(sb);                   // epilogue: [128][TT::STAGE_LD] FP32
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_tma[0], 1);
    mbar_init(&bar_tma[1], 1);
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TT::TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const size_t V = g.V, fs = V * 24;
  const long long ntiles = ((long long)V + S - 1) / S;
  uint32_t use[2] = {0, 0};
  int gc = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i0 = tile * S;
    for (int d = 0; d < 9; ++d) {
      const int b = gc & 1;
      // the MMAs that last read stage b must be complete before it is refilled
      if (use[b] > 0 && !mbar_wait(&bar_mma[b], (use[b] - 1) & 1, err)) fail = 1;
      __syncthreads();
      if (fail) break;
      if (tid == 0) {
        mbar_expect_tx(&bar_tma[b], TC_A_BYTES);
        bulk_load(abuf[b], Apack + (size_t)d * TC_M * TC_K, TC_A_BYTES, &bar_tma[b]);
      }
      // B_d: item (site q, input channel c) -> rows (4c .. 4c+3) re and (64 + 4c ..) im, columns 3q + colour
      const int dt = (ADJ && d > 0) ? (((d - 1) ^ 1) + 1) : d;
      for (int it = tid; it < S * 16; it += TC_THREADS) {
        const int q = it & (S - 1), c = it / S;
        const long long i = i0 + q;
        cplx<float> th[4][3];
        if (i < (long long)V) {
          const SiteRef s = decode(g, i);
          pt_transport(g, links, in + (size_t)c * fs, s, i, dt, th);
        } else {
#pragma unroll
          for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) th[sp][a] = {0.f, 0.f};
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int n = 3 * q + a;
          __nv_bfloat162 re01 = __floats2bfloat162_rn(th[0][a].re, th[1][a].re);
          __nv_bfloat162 re23 = __floats2bfloat162_rn(th[2][a].re, th[3][a].re);
          __nv_bfloat162 im01 = __floats2bfloat162_rn(th[0][a].im, th[1][a].im);
          __nv_bfloat162 im23 = __floats2bfloat162_rn(th[2][a].im, th[3][a].im);
          uint2 vr, vi;
          vr.x = *reinterpret_cast<uint32_t*>(&re01);
          vr.y = *reinterpret_cast<uint32_t*>(&re23);
          vi.x = *reinterpret_cast<uint32_t*>(&im01);
          vi.y = *reinterpret_cast<uint32_t*>(&im23);
          *reinterpret_cast<uint2*>(bbuf[b] + tc_off(n, 4 * c)) = vr;
          *reinterpret_cast<uint2*>(bbuf[b] + tc_off(n, 64 + 4 * c)) = vi;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // generic-proxy writes -> tensor core
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        if (mbar_wait(&bar_tma[b], use[b] & 1, err)) {
          const uint32_t a0 = smem_u32(abuf[b]), b0 = smem_u32(bbuf[b]);
#pragma unroll
          for (int kk = 0; kk < TC_K / 16; ++kk)
            tc_mma(tmem, tc_desc(a0 + kk * 256), tc_desc(b0 + kk * 256), TT::IDESC, (d > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&bar_mma[b]);
        } else {
          fail = 1;
        }
      }
      ++use[b];
      ++gc;
    }
    __syncthreads();
    if (fail) break;
    // epilogue: all MMAs of the tile complete -> TMEM rows to shared memory -> output fields
    const int bl = (gc - 1) & 1;
    if (!mbar_wait(&bar_mma[bl], (use[bl] - 1) & 1, err)) fail = 1;
    __syncthreads();
    if (fail) break;
    tc_fence_after();
    {
      const int row = 32 * (warp & 3) + lane, half = warp >> 2;
#pragma unroll
      for (int j = 0; j < TT::N / 2 / 16; ++j) {
        const int col = half * (TT::N / 2) + 16 * j;
        float v[16];
        tc_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) stage[row * TT::STAGE_LD + col + e] = v[e];
      }
    }
    tc_fence_before();
    __syncthreads();
    for (int it = tid; it < S * 16; it += TC_THREADS) {
      const int q = it & (S - 1), c = it / S;
      const long long i = i0 + q;
      if (i >= (long long)V) continue;
      cplx<float> o[12];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int m = 4 * c + sp, n = 3 * q + a;
          o[3 * sp + a] = {stage[m * TT::STAGE_LD + n], stage[(m + 64) * TT::STAGE_LD + n]};
        }
      store_site<float, 12>(out + (size_t)c * fs, V, i, o);
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TT::TMEM_COLS) : "memory");
}

// one 16 -> 16 layer (adjoint: W_d^+ and reversed transports) on the tensor cores
template <bool ADJ, int S>
static int launch_tc(dw_ctx* c, const __nv_bfloat16* A, const float* in, float* out, int* err, cudaStream_t st) {
  using TT = TcTile<S>;
  static bool attr_set = false;
  if (!attr_set) {
    DW_CUDA(cudaFuncSetAttribute(ptnet_tc_layer_kernel<ADJ, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TT::SMEM));
    attr_set = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (c->V + S - 1) / S;
  const unsigned grid = (unsigned)std::min<long long>(ntiles, (long long)sms * TT::MIN_BLOCKS);
  ptnet_tc_layer_kernel<ADJ, S><<<grid, TC_THREADS, TT::SMEM, st>>>(c->g, (const float*)c->links[DW_F32], A, in, out, err);
  dw_note_launch();
  return DW_OK;
}

// one 16 -> 16 layer (adjoint: W_d^+ and reversed transports) on the tensor cores; tiles of 64 sites
// (one CTA per SM) or, with DW_TC_TILE=32, of 32 sites (two CTAs per SM)
int tc_layer16(dw_ctx* c, const float2* W, int adjoint, const float* in, float* out, cudaStream_t st) {
  __nv_bfloat16* A = nullptr;
  int* err = nullptr;
  DW_CUDA(cudaMallocAsync((void**)&A, (size_t)9 * TC_A_BYTES, st));
  DW_CUDA(cudaMallocAsync((void**)&err, sizeof(int), st));
  DW_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int n = 9 * TC_M * TC_K;
  const char* te = getenv("DW_TC_TILE");
  const bool small = te && atoi(te) == 32;
  int rc;
  if (adjoint) {
    ptnet_tc_pack_kernel<true><<<(n + 255) / 256, 256, 0, st>>>(W, A); dw_note_launch();
    rc = small ? launch_tc<true, 32>(c, A, in, out, err, st) : launch_tc<true, 64>(c, A, in, out, err, st);
  } else {
    ptnet_tc_pack_kernel<false><<<(n + 255) / 256, 256, 0, st>>>(W, A); dw_note_launch();
    rc = small ? launch_tc<false, 32>(c, A, in, out, err, st) : launch_tc<false, 64>(c, A, in, out, err, st);
  }
  if (rc) return rc;
  DW_CUDA(cudaGetLastError());
  int herr = 0;
  DW_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DW_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(A, st);
  cudaFreeAsync(err, st);
  if (herr) { dw_set_error("ptnet tensor-core layer: a wait on the tensor core or bulk copy timed out"); return DW_ECUDA; }
  return DW_OK;
}

}  // namespace

extern "C" size_t ptnet_weight_count(int C) {
  return (size_t)9 * 16 * (C + C * C + C);   // complex numbers, layers 1 -> C -> C -> 1
}

static bool ptnet_ok(int C) { return C == 16; }

// acts: 2 * C fields (the two hidden layers), may be null for inference
static int ptnet_forward_impl(dw_ctx* c, int C, const float2* W, const float* x, float* y, float* acts,
                              cudaStream_t st) {
  const size_t fs = (size_t)c->V * 24;
  float* h1 = acts;
  float* own = nullptr;
  if (!h1) {
    DW_CUDA(cudaMalloc(&own, 2 * C * fs * sizeof(float)));
    h1 = own;
  }
  float* h2 = h1 + (size_t)C * fs;
  const size_t w1 = 9 * 16 * C, w2 = 9 * 16 * C * C;
  launch_layer<1, 16, false>(c, W, x, h1, st);
  launch_layer<16, 16, false>(c, W + w1, h1, h2, st);
  launch_layer<16, 1, false>(c, W + w1 + w2, h2, y, st);
  cudaError_t e = cudaGetLastError();
  if (own) {
    cudaStreamSynchronize(st);
    cudaFree(own);
  }
  if (e != cudaSuccess) return dw_cuda_fail(e, "ptnet_forward");
  return DW_OK;
}

extern "C" int ptnet_forward(dw_ctx* c, int C, const void* W, int nf, const void* x, void* y, void* stream) {
  if (!c || !W || !x || !y || x == y || nf < 1 || !ptnet_ok(C)) {
    dw_set_error("ptnet_forward: bad argument (C must be 16)");
    return DW_EINVAL;
  }
  const size_t fs = (size_t)c->V * 24;
  float* acts = nullptr;
  DW_CUDA(cudaMalloc(&acts, 2 * C * fs * sizeof(float)));
  int rc = DW_OK;
  for (int f = 0; f < nf && rc == DW_OK; ++f)
    rc = ptnet_forward_impl(c, C, (const float2*)W, (const float*)x + f * fs, (float*)y + f * fs, acts,
                            (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  cudaFree(acts);
  return rc;
}

// One 16 -> 16 layer on a set of 16 channel fields: out = sum_d W_d T_d in (adjoint:
// sum_d W_d^+ T_d^+ in), on the tensor cores (BF16 operands, FP32 accumulation) or the CUDA cores (FP32).
extern "C" int ptnet_layer16(dw_ctx* c, const void* W, int adjoint, int tensor_cores, const void* in, void* out,
                             void* stream) {
  if (!c || !W || !in || !out || in == out) { dw_set_error("ptnet_layer16: bad argument"); return DW_EINVAL; }
  if (int rc = dw_check_device(c, "ptnet_layer16")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (tensor_cores) return tc_layer16(c, (const float2*)W, adjoint, (const float*)in, (float*)out, st);
  if (adjoint) launch_layer<16, 16, true>(c, (const float2*)W, (const float*)in, (float*)out, st);
  else launch_layer<16, 16, false>(c, (const float2*)W, (const float*)in, (float*)out, st);
  DW_CUDA(cudaGetLastError());
  DW_CUDA(cudaStreamSynchronize(st));
  return DW_OK;
}

// The network with its 16 -> 16 layer on the tensor cores (the 1 -> 16 and 16 -> 1 layers, 16x fewer
// flops, on the CUDA cores).
extern "C" int ptnet_forward_tc(dw_ctx* c, int C, const void* Wv, int nf, const void* x, void* y, void* stream) {
  if (!c || !Wv || !x || !y || x == y || nf < 1 || !ptnet_ok(C)) {
    dw_set_error("ptnet_forward_tc: bad argument (C must be 16)");
    return DW_EINVAL;
  }
  if (int rc = dw_check_device(c, "ptnet_forward_tc")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* W = (const float2*)Wv;
  const size_t fs = (size_t)c->V * 24, w1 = 9 * 16 * C, w2 = 9 * 16 * C * C;
  float* acts = nullptr;
  DW_CUDA(cudaMalloc(&acts, 2 * C * fs * sizeof(float)));
  float* h1 = acts;
  float* h2 = acts + (size_t)C * fs;
  int rc = DW_OK;
  for (int f = 0; f < nf && rc == DW_OK; ++f) {
    launch_layer<1, 16, false>(c, W, (const float*)x + f * fs, h1, st);
    rc = tc_layer16(c, W + w1, 0, h1, h2, st);
    if (rc == DW_OK) launch_layer<16, 1, false>(c, W + w1 + w2, h2, (float*)y + f * fs, st);
  }
  cudaStreamSynchronize(st);
  cudaFree(acts);
  if (rc == DW_OK) DW_CUDA(cudaGetLastError());
  return rc;
}

// loss = sum_f |N(x_f) - y_f|^2 / sum_f |y_f|^2 and its gradient dL/dRe W + i dL/dIm W
extern "C" int ptnet_loss_grad(dw_ctx* c, int C, const void* Wv, int nf, const void* xv, const void* yv,
                               void* gradv, double* loss, void* stream) {
  if (!c || !Wv || !xv || !yv || !gradv || nf < 1 || !ptnet_ok(C)) {
    dw_set_error("ptnet_loss_grad: bad argument (C must be 16)");
    return DW_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float2* W = (const float2*)Wv;
  const size_t fs = (size_t)c->V * 24, n = (size_t)c->V * 12;
  const size_t w1 = 9 * 16 * C, w2 = 9 * 16 * C * C, w3 = 9 * 16 * C, nw = w1 + w2 + w3;
  const long long chunk = 4096;
  const int nchunk = (int)((c->V + chunk - 1) / chunk);
  float *acts = nullptr, *out = nullptr, *g2 = nullptr, *g1 = nullptr;
  float2 *partial = nullptr, *gacc = nullptr, *gtmp = nullptr;
  std::vector<void*> owned;
  auto al = [&](void** p, size_t b) -> int {
    cudaError_t e = cudaMalloc(p, b);
    if (e != cudaSuccess) return dw_cuda_fail(e, "cudaMalloc");
    owned.push_back(*p);
    return DW_OK;
  };
  int rc;
  if ((rc = al((void**)&acts, 2 * C * fs * sizeof(float))) || (rc = al((void**)&out, fs * sizeof(float))) ||
      (rc = al((void**)&g2, C * fs * sizeof(float))) || (rc = al((void**)&g1, C * fs * sizeof(float))) ||
      (rc = al((void**)&partial, (size_t)nchunk * 9 * 16 * C * C * sizeof(float2))) ||
      (rc = al((void**)&gacc, nw * sizeof(float2))) || (rc = al((void**)&gtmp, nw * sizeof(float2)))) {
    for (void* p : owned) cudaFree(p);
    return rc;
  }
  float* h1 = acts;
  float* h2 = acts + (size_t)C * fs;
  DW_CUDA(cudaMemsetAsync(gacc, 0, nw * sizeof(float2), st));
  double num = 0, den = 0;
  std::vector<double> hh(3);
  for (int f = 0; f < nf; ++f) {
    const float* x = (const float*)xv + f * fs;
    const float* y = (const float*)yv + f * fs;
    if ((rc = ptnet_forward_impl(c, C, W, x, out, acts, st))) break;
    // e = out - y ; loss numerator |e|^2, denominator |y|^2
    blas_axpy<float>(y, out, -1.0, 0.0, n, st);
    double* dres = c->d_red + 65536 + 12288;
    blas_dot<float>(c, out, out, n, dres, st);
    blas_dot<float>(c, y, y, n, dres + 3, st);
    // back-propagation: gradient of |e|^2 wrt the output is 2 e
    const dim3 g3(nchunk, 9);
    ptnet_dw_kernel<16, 1><<<g3, 256, 0, st>>>(c->g, (const float*)c->links[DW_F32], out, h2, partial, chunk); dw_note_launch();
    ptnet_dw_reduce_kernel<<<(unsigned)((9 * 16 * C + 255) / 256), 256, 0, st>>>(partial, nchunk, 16 * C, 2.f,
                                                                               gtmp + w1 + w2); dw_note_launch();
    launch_layer<16, 1, true>(c, W + w1 + w2, out, g2, st);
    ptnet_dw_kernel<16, 16><<<g3, 256, 0, st>>>(c->g, (const float*)c->links[DW_F32], g2, h1, partial, chunk); dw_note_launch();
    ptnet_dw_reduce_kernel<<<(unsigned)((9 * 16 * C * C + 255) / 256), 256, 0, st>>>(partial, nchunk, 16 * C * C,
                                                                                   2.f, gtmp + w1); dw_note_launch();
    launch_layer<16, 16, true>(c, W + w1, g2, g1, st);
    ptnet_dw_kernel<1, 16><<<g3, 256, 0, st>>>(c->g, (const float*)c->links[DW_F32], g1, x, partial, chunk); dw_note_launch();
    ptnet_dw_reduce_kernel<<<(unsigned)((9 * 16 * C + 255) / 256), 256, 0, st>>>(partial, nchunk, 16 * C, 2.f,
                                                                               gtmp); dw_note_launch();
    blas_axpy<float>((const float*)gtmp, (float*)gacc, 1.0, 0.0, nw, st);
    cudaError_t e = cudaMemcpyAsync(c->h_red, dres, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc = dw_cuda_fail(e, "ptnet_loss_grad"); break; }
    num += c->h_red[2];
    den += c->h_red[5];
  }
  if (!rc) {
    // normalise by sum |y|^2
    blas_scale<float>((float*)gacc, den > 0 ? 1.0 / den : 0.0, 0.0, nw, st);
    cudaMemcpyAsync(gradv, gacc, nw * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    if (loss) *loss = den > 0 ? num / den : 0.0;
  }
  for (void* p : owned) cudaFree(p);
  return rc;
}

extern "C" int ptnet_adam(size_t ncomplex, void* W, const void* grad, void* m, void* v, int step, double lr,
                          void* stream) {
  if (!W || !grad || !m || !v || step < 1) { dw_set_error("ptnet_adam: bad argument"); return DW_EINVAL; }
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  const size_t n = 2 * ncomplex;
  ptnet_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      n, (float*)W, (const float*)grad, (float*)m, (float*)v, (float)lr, b1, b2, 1e-8f, c1, c2); dw_note_launch();
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

// the plain procedure (5.1) on nf packed FP32 fields in place: nsteps x (psi <- M_sap psi / |.|)
extern "C" int dfl_inverse_iteration(dw_ctx* c, int ncy, int nmr, int nsteps, int nf, void* fields, void* stream) {
  if (!c || !fields || nf < 1 || nsteps < 0) { dw_set_error("dfl_inverse_iteration: bad argument"); return DW_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t fs = (size_t)c->V * 24, n = (size_t)c->V * 12;
  float* tmp = nullptr;
  DW_CUDA(cudaMalloc(&tmp, fs * nf * sizeof(float)));
  float* f = (float*)fields;
  double* dres = c->d_red + 65536 + 16384;
  int rc = DW_OK;
  for (int it = 0; it < nsteps && rc == DW_OK; ++it) {
    rc = nf > 1 ? sap_apply_mrhs(c, ncy, nmr, f, tmp, nf, st) : sap_apply<float>(c, ncy, nmr, f, tmp, st);
    if (rc) break;
    for (int l = 0; l < nf; ++l) blas_dot<float>(c, tmp + l * fs, tmp + l * fs, n, dres + 3 * l, st);
    cudaError_t e = cudaMemcpyAsync(c->h_red, dres, 3 * nf * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc = dw_cuda_fail(e, "dfl_inverse_iteration"); break; }
    for (int l = 0; l < nf; ++l) blas_convert<float, float>(tmp + l * fs, f + l * fs, 1.0 / sqrt(c->h_red[3 * l + 2]), n, st);
  }
  cudaStreamSynchronize(st);
  cudaFree(tmp);
  return rc;
}
