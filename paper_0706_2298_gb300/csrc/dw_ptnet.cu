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
