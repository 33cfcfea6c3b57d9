// Training and inference kernels of the sweep surrogate (include/hlb_surrogate.h).
// Small FP32 network: three strided conv1d layers over the early wall-flux
// history, mean pooling, and a three-layer MLP.  Batches are at most a few
// hundred samples, so plain SIMT kernels (shared-memory tiled for the linear
// layers) are used; every step of forward, backward and Adam runs here.
#include <math.h>
#include <stdint.h>

#include "hlb_surrogate.h"

#include <cuda_runtime.h>

namespace {

struct Dims {
  int L0, C1, C2, C3, K, S, NS, H, NOUT, L1, L2, L3;
};

bool dims_of(const hlb_sur_config* c, Dims* d) {
  if (!c) return false;
  if (c->L0 < 1 || c->C1 < 1 || c->C2 < 1 || c->C3 < 1 || c->K < 1 || c->S < 1 || c->NS < 0 || c->H < 1 ||
      c->NOUT < 2)
    return false;
  d->L0 = c->L0; d->C1 = c->C1; d->C2 = c->C2; d->C3 = c->C3; d->K = c->K; d->S = c->S;
  d->NS = c->NS; d->H = c->H; d->NOUT = c->NOUT;
  if (c->L0 < c->K) return false;
  d->L1 = (c->L0 - c->K) / c->S + 1;
  if (d->L1 < c->K) return false;
  d->L2 = (d->L1 - c->K) / c->S + 1;
  if (d->L2 < c->K) return false;
  d->L3 = (d->L2 - c->K) / c->S + 1;
  return true;
}

struct Offsets {  // parameter offsets (floats)
  size_t W1, b1, W2, b2, W3, b3, F1, c1, F2, c2, F3, c3, total;
};

Offsets param_offsets(const Dims& d) {
  Offsets o;
  size_t p = 0;
  o.W1 = p; p += (size_t)d.C1 * d.K;
  o.b1 = p; p += d.C1;
  o.W2 = p; p += (size_t)d.C2 * d.C1 * d.K;
  o.b2 = p; p += d.C2;
  o.W3 = p; p += (size_t)d.C3 * d.C2 * d.K;
  o.b3 = p; p += d.C3;
  o.F1 = p; p += (size_t)d.H * (d.C3 + d.NS);
  o.c1 = p; p += d.H;
  o.F2 = p; p += (size_t)d.H * d.H;
  o.c2 = p; p += d.H;
  o.F3 = p; p += (size_t)d.NOUT * d.H;
  o.c3 = p; p += d.NOUT;
  o.total = p;
  return o;
}

size_t al(size_t n) { return (n + 63) & ~(size_t)63; }  // 256-byte aligned float counts

struct Acts {  // workspace offsets (floats)
  size_t z1, a1, z2, a2, z3, a3, h0, z4, a4, z5, a5, y, dy, dz5, dz4, dh0, dz3, dz2, dz1, loss, total;
};

Acts act_offsets(const Dims& d, int B) {
  Acts a;
  size_t p = 0;
  const size_t n1 = (size_t)B * d.C1 * d.L1, n2 = (size_t)B * d.C2 * d.L2, n3 = (size_t)B * d.C3 * d.L3;
  const size_t nh0 = (size_t)B * (d.C3 + d.NS), nh = (size_t)B * d.H, ny = (size_t)B * d.NOUT;
  a.z1 = p; p += al(n1);
  a.a1 = p; p += al(n1);
  a.z2 = p; p += al(n2);
  a.a2 = p; p += al(n2);
  a.z3 = p; p += al(n3);
  a.a3 = p; p += al(n3);
  a.h0 = p; p += al(nh0);
  a.z4 = p; p += al(nh);
  a.a4 = p; p += al(nh);
  a.z5 = p; p += al(nh);
  a.a5 = p; p += al(nh);
  a.y = p; p += al(ny);
  a.dy = p; p += al(ny);
  a.dz5 = p; p += al(nh);
  a.dz4 = p; p += al(nh);
  a.dh0 = p; p += al(nh0);
  a.dz3 = p; p += al(n3);
  a.dz2 = p; p += al(n2);
  a.dz1 = p; p += al(n1);
  a.loss = p; p += al(2);
  a.total = p;
  return a;
}

// z[b,o,t] = bias[o] + sum_{c,k} W[o,c,k] x[b,c,S t + k];  a = max(z, 0)
__global__ void k_conv_fwd(const float* __restrict__ x, int Cin, int Lin, const float* __restrict__ W,
                           const float* __restrict__ bias, int Cout, int K, int S, int Lout, int B,
                           float* __restrict__ z, float* __restrict__ a) {
  const long long n = (long long)B * Cout * Lout;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e % Lout);
    const int o = (int)((e / Lout) % Cout);
    const int b = (int)(e / ((long long)Lout * Cout));
    float s = bias[o];
    const float* xb = x + (long long)b * Cin * Lin + (long long)S * t;
    const float* wo = W + (long long)o * Cin * K;
    for (int c = 0; c < Cin; ++c)
      for (int k = 0; k < K; ++k) s += wo[c * K + k] * xb[(long long)c * Lin + k];
    z[e] = s;
    a[e] = fmaxf(s, 0.f);
  }
}

// dx[b,c,u] = sum over (o, k, t) with S t + k = u of W[o,c,k] dz[b,o,t]; times (zprev > 0)
__global__ void k_conv_bwd_data(const float* __restrict__ dz, const float* __restrict__ W, int B, int Cin, int Lin,
                                int Cout, int K, int S, int Lout, const float* __restrict__ zprev,
                                float* __restrict__ dx) {
  const long long n = (long long)B * Cin * Lin;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e % Lin);
    const int c = (int)((e / Lin) % Cin);
    const int b = (int)(e / ((long long)Lin * Cin));
    float s = 0.f;
    for (int k = 0; k < K; ++k) {
      const int v = u - k;
      if (v < 0 || v % S != 0) continue;
      const int t = v / S;
      if (t >= Lout) continue;
      for (int o = 0; o < Cout; ++o) s += W[((long long)o * Cin + c) * K + k] * dz[((long long)b * Cout + o) * Lout + t];
    }
    dx[e] = zprev ? (zprev[e] > 0.f ? s : 0.f) : s;
  }
}

template <int NT>
__device__ __forceinline__ float block_sum(float v) {
  __shared__ float red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

// One block per weight (o, c, k): dW = sum_{b,t} dz[b,o,t] x[b,c,S t + k];
// the last Cout blocks compute db[o] = sum_{b,t} dz[b,o,t].
__global__ void __launch_bounds__(256) k_conv_bwd_w(const float* __restrict__ dz, const float* __restrict__ x, int B,
                                                    int Cin, int Lin, int Cout, int K, int S, int Lout,
                                                    float* __restrict__ dW, float* __restrict__ db) {
  const int nw = Cout * Cin * K;
  const int id = blockIdx.x;
  const long long n = (long long)B * Lout;
  float s = 0.f;
  if (id < nw) {
    const int k = id % K, c = (id / K) % Cin, o = id / (K * Cin);
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const int t = (int)(e % Lout), b = (int)(e / Lout);
      s += dz[((long long)b * Cout + o) * Lout + t] * x[((long long)b * Cin + c) * Lin + (long long)S * t + k];
    }
    s = block_sum<256>(s);
    if (threadIdx.x == 0) dW[id] = s;
  } else {
    const int o = id - nw;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const int t = (int)(e % Lout), b = (int)(e / Lout);
      s += dz[((long long)b * Cout + o) * Lout + t];
    }
    s = block_sum<256>(s);
    if (threadIdx.x == 0) db[o] = s;
  }
}

// h0[b, c] = mean_t a[b, c, t] for c < C; h0[b, C + j] = scal[b, j]
__global__ void k_pool_concat(const float* __restrict__ a, int B, int C, int L, const float* __restrict__ scal, int NS,
                              float* __restrict__ h0) {
  const int W = C + NS;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * W; e += gridDim.x * blockDim.x) {
    const int b = e / W, c = e % W;
    if (c < C) {
      float s = 0.f;
      const float* p = a + ((long long)b * C + c) * L;
      for (int t = 0; t < L; ++t) s += p[t];
      h0[e] = s / (float)L;
    } else {
      h0[e] = scal[b * NS + (c - C)];
    }
  }
}

// dz3[b,c,t] = dh0[b,c] / L * (z3 > 0)
__global__ void k_pool_bwd(const float* __restrict__ dh0, int ldh, const float* __restrict__ z, int B, int C, int L,
                           float* __restrict__ dzo) {
  const long long n = (long long)B * C * L;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)((e / L) % C), b = (int)(e / ((long long)L * C));
    dzo[e] = z[e] > 0.f ? dh0[(long long)b * ldh + c] / (float)L : 0.f;
  }
}

constexpr int TL = 16;

// z[b,n] = bias[n] + sum_k x[b,k] F[n,k]; a = relu(z) (if a != null).  16x16 tiles.
__global__ void k_linear_fwd(const float* __restrict__ x, int B, int Nin, const float* __restrict__ F,
                             const float* __restrict__ bias, int Nout, float* __restrict__ z, float* __restrict__ a) {
  __shared__ float xs[TL][TL + 1], fs[TL][TL + 1];
  const int b = blockIdx.y * TL + threadIdx.y;
  const int n = blockIdx.x * TL + threadIdx.x;
  float s = 0.f;
  for (int k0 = 0; k0 < Nin; k0 += TL) {
    const int kx = k0 + threadIdx.x;
    xs[threadIdx.y][threadIdx.x] = (b < B && kx < Nin) ? x[(long long)b * Nin + kx] : 0.f;
    const int nf = blockIdx.x * TL + threadIdx.y;
    fs[threadIdx.y][threadIdx.x] = (nf < Nout && kx < Nin) ? F[(long long)nf * Nin + kx] : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TL; ++kk) s += xs[threadIdx.y][kk] * fs[threadIdx.x][kk];
    __syncthreads();
  }
  if (b < B && n < Nout) {
    s += bias[n];
    z[(long long)b * Nout + n] = s;
    if (a) a[(long long)b * Nout + n] = fmaxf(s, 0.f);
  }
}

// dx[b,k] = sum_n dz[b,n] F[n,k], times (zprev[b,k] > 0) if zprev != null
__global__ void k_linear_bwd_data(const float* __restrict__ dz, int B, int Nout, const float* __restrict__ F, int Nin,
                                  const float* __restrict__ zprev, float* __restrict__ dx) {
  __shared__ float ds[TL][TL + 1], fs[TL][TL + 1];
  const int b = blockIdx.y * TL + threadIdx.y;
  const int k = blockIdx.x * TL + threadIdx.x;
  float s = 0.f;
  for (int n0 = 0; n0 < Nout; n0 += TL) {
    const int nx = n0 + threadIdx.x;
    ds[threadIdx.y][threadIdx.x] = (b < B && nx < Nout) ? dz[(long long)b * Nout + nx] : 0.f;
    const int ny = n0 + threadIdx.y;
    fs[threadIdx.y][threadIdx.x] = (ny < Nout && k < Nin) ? F[(long long)ny * Nin + k] : 0.f;
    __syncthreads();
#pragma unroll
    for (int nn = 0; nn < TL; ++nn) s += ds[threadIdx.y][nn] * fs[nn][threadIdx.x];
    __syncthreads();
  }
  if (b < B && k < Nin) {
    const long long e = (long long)b * Nin + k;
    dx[e] = zprev ? (zprev[e] > 0.f ? s : 0.f) : s;
  }
}

// dF[n,k] = sum_b dz[b,n] x[b,k]; dc[n] = sum_b dz[b,n] (column k = Nin of the grid)
__global__ void k_linear_bwd_w(const float* __restrict__ dz, const float* __restrict__ x, int B, int Nout, int Nin,
                               float* __restrict__ dF, float* __restrict__ dc) {
  __shared__ float ds[TL][TL + 1], xs[TL][TL + 1];
  const int n = blockIdx.y * TL + threadIdx.y;
  const int k = blockIdx.x * TL + threadIdx.x;
  float s = 0.f;
  for (int b0 = 0; b0 < B; b0 += TL) {
    const int bx = b0 + threadIdx.x;
    const int nd = blockIdx.y * TL + threadIdx.y;
    ds[threadIdx.y][threadIdx.x] = (bx < B && nd < Nout) ? dz[(long long)bx * Nout + nd] : 0.f;
    const int by = b0 + threadIdx.y;
    xs[threadIdx.y][threadIdx.x] =
        (by < B && k < Nin + 1) ? (k < Nin ? x[(long long)by * Nin + k] : 1.f) : 0.f;
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < TL; ++bb) s += ds[threadIdx.y][bb] * xs[bb][threadIdx.x];
    __syncthreads();
  }
  if (n < Nout) {
    if (k < Nin) dF[(long long)n * Nin + k] = s;
    else if (k == Nin) dc[n] = s;
  }
}

// Loss terms and dL/dy (one block; B <= blockDim.x * iterations).
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ y, int B, int NOUT,
                                              const float* __restrict__ target, const int* __restrict__ label,
                                              float* __restrict__ dy, float* __restrict__ loss) {
  float mse = 0.f, ce = 0.f;
  const float invB = 1.f / (float)B;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float* yb = y + (long long)b * NOUT;
    float* db = dy + (long long)b * NOUT;
    const float r = yb[0] - target[b];
    mse += r * r;
    db[0] = 2.f * r * invB;
    float m = yb[1];
    for (int q = 2; q < NOUT; ++q) m = fmaxf(m, yb[q]);
    float se = 0.f;
    for (int q = 1; q < NOUT; ++q) se += expf(yb[q] - m);
    const int lb = label[b];
    ce += logf(se) + m - yb[1 + lb];
    for (int q = 1; q < NOUT; ++q) db[q] = (expf(yb[q] - m) / se - (q - 1 == lb ? 1.f : 0.f)) * invB;
  }
  mse = block_sum<256>(mse);
  __syncthreads();
  ce = block_sum<256>(ce);
  if (threadIdx.x == 0) {
    loss[0] = mse * invB;
    loss[1] = ce * invB;
  }
}

__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

bool ws_ok(const Dims& d, int B, void* ws, size_t bytes) {
  if (!ws || ((uintptr_t)ws & 255)) return false;
  return bytes >= act_offsets(d, B).total * sizeof(float);
}

void forward(const Dims& d, const Offsets& o, const Acts& A, const float* P, const float* hist, const float* scal,
             int B, float* w, cudaStream_t s) {
  k_conv_fwd<<<grid_for((long long)B * d.C1 * d.L1), 256, 0, s>>>(hist, 1, d.L0, P + o.W1, P + o.b1, d.C1, d.K, d.S,
                                                                  d.L1, B, w + A.z1, w + A.a1);
  k_conv_fwd<<<grid_for((long long)B * d.C2 * d.L2), 256, 0, s>>>(w + A.a1, d.C1, d.L1, P + o.W2, P + o.b2, d.C2, d.K,
                                                                  d.S, d.L2, B, w + A.z2, w + A.a2);
  k_conv_fwd<<<grid_for((long long)B * d.C3 * d.L3), 256, 0, s>>>(w + A.a2, d.C2, d.L2, P + o.W3, P + o.b3, d.C3, d.K,
                                                                  d.S, d.L3, B, w + A.z3, w + A.a3);
  const int W0 = d.C3 + d.NS;
  k_pool_concat<<<grid_for((long long)B * W0), 256, 0, s>>>(w + A.a3, B, d.C3, d.L3, scal, d.NS, w + A.h0);
  const dim3 blk(TL, TL);
  k_linear_fwd<<<dim3((d.H + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.h0, B, W0, P + o.F1, P + o.c1, d.H,
                                                                            w + A.z4, w + A.a4);
  k_linear_fwd<<<dim3((d.H + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.a4, B, d.H, P + o.F2, P + o.c2, d.H,
                                                                            w + A.z5, w + A.a5);
  k_linear_fwd<<<dim3((d.NOUT + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.a5, B, d.H, P + o.F3, P + o.c3,
                                                                               d.NOUT, w + A.y, nullptr);
}

}  // namespace

extern "C" {

void hlb_sur_config_default(hlb_sur_config* c) {
  if (!c) return;
  c->L0 = 500;
  c->C1 = 16;
  c->C2 = 32;
  c->C3 = 32;
  c->K = 5;
  c->S = 2;
  c->NS = 2;
  c->H = 256;
  c->NOUT = 6;
}

size_t hlb_sur_param_count(const hlb_sur_config* c) {
  Dims d;
  if (!dims_of(c, &d)) return 0;
  return param_offsets(d).total;
}

size_t hlb_sur_workspace_bytes(const hlb_sur_config* c, int B) {
  Dims d;
  if (!dims_of(c, &d) || B < 1 || B > 4096) return 0;
  return act_offsets(d, B).total * sizeof(float);
}

hlb_status hlb_sur_forward(const hlb_sur_config* c, const float* d_params, const float* d_hist, const float* d_scal,
                           int B, float* d_out, void* d_ws, size_t ws_bytes, void* stream) {
  Dims d;
  if (!dims_of(c, &d) || B < 1 || B > 4096 || !d_params || !d_hist || (d.NS > 0 && !d_scal) || !d_out)
    return HLB_EINVAL;
  if (!ws_ok(d, B, d_ws, ws_bytes)) return HLB_EINVAL;
  const Offsets o = param_offsets(d);
  const Acts A = act_offsets(d, B);
  float* w = (float*)d_ws;
  cudaStream_t s = (cudaStream_t)stream;
  forward(d, o, A, d_params, d_hist, d_scal, B, w, s);
  if (cudaMemcpyAsync(d_out, w + A.y, sizeof(float) * (size_t)B * d.NOUT, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HLB_ECUDA;
  return cudaGetLastError() == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

hlb_status hlb_sur_loss_grad(const hlb_sur_config* c, const float* d_params, const float* d_hist,
                             const float* d_scal, const float* d_target, const int* d_label, int B, float* d_grad,
                             float* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
  Dims d;
  if (!dims_of(c, &d) || B < 1 || B > 4096 || !d_params || !d_hist || (d.NS > 0 && !d_scal) || !d_target ||
      !d_label || !d_grad || !d_loss)
    return HLB_EINVAL;
  if (!ws_ok(d, B, d_ws, ws_bytes)) return HLB_EINVAL;
  const Offsets o = param_offsets(d);
  const Acts A = act_offsets(d, B);
  float* w = (float*)d_ws;
  const float* P = d_params;
  float* G = d_grad;
  cudaStream_t s = (cudaStream_t)stream;
  forward(d, o, A, P, d_hist, d_scal, B, w, s);
  k_loss<<<1, 256, 0, s>>>(w + A.y, B, d.NOUT, d_target, d_label, w + A.dy, w + A.loss);
  const dim3 blk(TL, TL);
  const int W0 = d.C3 + d.NS;
  // layer 6 (output)
  k_linear_bwd_w<<<dim3((d.H + 1 + TL - 1) / TL, (d.NOUT + TL - 1) / TL), blk, 0, s>>>(w + A.dy, w + A.a5, B, d.NOUT,
                                                                                      d.H, G + o.F3, G + o.c3);
  k_linear_bwd_data<<<dim3((d.H + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.dy, B, d.NOUT, P + o.F3, d.H,
                                                                                w + A.z5, w + A.dz5);
  // layer 5
  k_linear_bwd_w<<<dim3((d.H + 1 + TL - 1) / TL, (d.H + TL - 1) / TL), blk, 0, s>>>(w + A.dz5, w + A.a4, B, d.H, d.H,
                                                                                   G + o.F2, G + o.c2);
  k_linear_bwd_data<<<dim3((d.H + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.dz5, B, d.H, P + o.F2, d.H,
                                                                                w + A.z4, w + A.dz4);
  // layer 4
  k_linear_bwd_w<<<dim3((W0 + 1 + TL - 1) / TL, (d.H + TL - 1) / TL), blk, 0, s>>>(w + A.dz4, w + A.h0, B, d.H, W0,
                                                                                  G + o.F1, G + o.c1);
  k_linear_bwd_data<<<dim3((W0 + TL - 1) / TL, (B + TL - 1) / TL), blk, 0, s>>>(w + A.dz4, B, d.H, P + o.F1, W0,
                                                                               nullptr, w + A.dh0);
  // pooling and conv layers
  k_pool_bwd<<<grid_for((long long)B * d.C3 * d.L3), 256, 0, s>>>(w + A.dh0, W0, w + A.z3, B, d.C3, d.L3, w + A.dz3);
  k_conv_bwd_w<<<d.C3 * d.C2 * d.K + d.C3, 256, 0, s>>>(w + A.dz3, w + A.a2, B, d.C2, d.L2, d.C3, d.K, d.S, d.L3,
                                                        G + o.W3, G + o.b3);
  k_conv_bwd_data<<<grid_for((long long)B * d.C2 * d.L2), 256, 0, s>>>(w + A.dz3, P + o.W3, B, d.C2, d.L2, d.C3, d.K,
                                                                      d.S, d.L3, w + A.z2, w + A.dz2);
  k_conv_bwd_w<<<d.C2 * d.C1 * d.K + d.C2, 256, 0, s>>>(w + A.dz2, w + A.a1, B, d.C1, d.L1, d.C2, d.K, d.S, d.L2,
                                                        G + o.W2, G + o.b2);
  k_conv_bwd_data<<<grid_for((long long)B * d.C1 * d.L1), 256, 0, s>>>(w + A.dz2, P + o.W2, B, d.C1, d.L1, d.C2, d.K,
                                                                      d.S, d.L2, w + A.z1, w + A.dz1);
  k_conv_bwd_w<<<d.C1 * 1 * d.K + d.C1, 256, 0, s>>>(w + A.dz1, d_hist, B, 1, d.L0, d.C1, d.K, d.S, d.L1, G + o.W1,
                                                     G + o.b1);
  if (cudaMemcpyAsync(d_loss, w + A.loss, 2 * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HLB_ECUDA;
  return cudaGetLastError() == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

hlb_status hlb_sur_adam(long long n, float* d_params, const float* d_grad, float* d_m, float* d_v, float lr,
                        float beta1, float beta2, float eps, int t, void* stream) {
  if (n < 1 || !d_params || !d_grad || !d_m || !d_v || t < 1) return HLB_EINVAL;
  const float bc1 = 1.f - powf(beta1, (float)t);
  const float bc2 = 1.f - powf(beta2, (float)t);
  k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, d_params, d_grad, d_m, d_v, lr, beta1, beta2, eps, bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

}  // extern "C"
