// unet.cu -- learned warm start for the pair Poisson solves.
//
// A 3-level 3D U-Net maps a pair's right-hand side b (4 pi rho plus the
// ghost-shell boundary terms, the same b the CG solves A v = b with) and
// the box mask, embedded at the centre of a 32^3 patch, to an initial guess
// v0 for the CG.  The problem is linear in b, so the patch input is b / s
// and the output is scaled back by s, s = max |b| over the box.  The CG
// then starts from v0 and runs to the same tolerance as from zero; only
// its iteration count changes.
//
// Network (width c): conv3(2 -> c) relu, conv3(c -> c) relu [skip 1],
// avg-pool 2, conv3(c -> 2c) relu, conv3(2c -> 2c) relu [skip 2],
// avg-pool 2, conv3(2c -> 4c) relu, conv3(4c -> 4c) relu, nearest up 2,
// concat skip 2, conv3(6c -> 2c) relu, conv3(2c -> 2c) relu, nearest up 2,
// concat skip 1, conv3(3c -> c) relu, conv3(c -> c) relu, conv1(c -> 1).
// conv3 = 3x3x3 with zero padding.  Weights are BF16 (an FP32 master copy
// for the optimizer), activations and accumulation FP32.  Training: masked
// mean squared error against the CG solution, Adam.  All reductions run in
// a fixed order (no floating-point atomics), so training is deterministic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "sea_internal.cuh"

#define UN_P 32                         // patch edge
#define UN_V (UN_P * UN_P * UN_P)       // patch points

namespace sea {
namespace {

__device__ __forceinline__ int vox(int z, int y, int x, int D) { return (z * D + y) * D + x; }

// y[b][yc0 + co][p] = act(bias[co] + sum_ci sum_k w[co][ci][k] x[b][xc0 + ci][p + off(k)])
// over a D^3 volume.  CTA: 4 x 8 x 8 output voxels (one per thread) x 8
// output channels; per input channel the 6 x 10 x 10 input halo and the
// 8 x 27 weights sit in shared memory.
#define CV_CO 8
__global__ void __launch_bounds__(256)
    k_conv3(const float* __restrict__ x, int xC, int xc0, int Cin,
            const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
            float* __restrict__ y, int yC, int yc0, int Cout, int D, int relu) {
  __shared__ float sx[6][10][10];
  __shared__ float sw[CV_CO][27];
  const int tiles_x = (D + 7) / 8, tiles_y = (D + 7) / 8;
  const int tile = blockIdx.x;
  const int tx0 = (tile % tiles_x) * 8, ty0 = ((tile / tiles_x) % tiles_y) * 8,
            tz0 = (tile / (tiles_x * tiles_y)) * 4;
  const int co0 = blockIdx.y * CV_CO, b = blockIdx.z;
  const int lx = threadIdx.x % 8, ly = (threadIdx.x / 8) % 8, lz = threadIdx.x / 64;
  const int ox = tx0 + lx, oy = ty0 + ly, oz = tz0 + lz;
  float acc[CV_CO];
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) acc[c] = (bias && co0 + c < Cout) ? bias[co0 + c] : 0.f;
  const size_t V = (size_t)D * D * D;
  for (int ci = 0; ci < Cin; ++ci) {
    __syncthreads();
    const float* xs = x + ((size_t)b * xC + xc0 + ci) * V;
    for (int q = threadIdx.x; q < 600; q += blockDim.x) {
      const int hx = q % 10, hy = (q / 10) % 10, hz = q / 100;
      const int gx = tx0 + hx - 1, gy = ty0 + hy - 1, gz = tz0 + hz - 1;
      sx[hz][hy][hx] = (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D)
                           ? xs[vox(gz, gy, gx, D)]
                           : 0.f;
    }
    for (int q = threadIdx.x; q < CV_CO * 27; q += blockDim.x) {
      const int c = q / 27, k = q % 27;
      sw[c][k] = co0 + c < Cout ? __bfloat162float(w[((size_t)(co0 + c) * Cin + ci) * 27 + k]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const float xv = sx[lz + k / 9][ly + (k / 3) % 3][lx + k % 3];
#pragma unroll
      for (int c = 0; c < CV_CO; ++c) acc[c] = fmaf(sw[c][k], xv, acc[c]);
    }
  }
  if (ox >= D || oy >= D || oz >= D) return;
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) {
    if (co0 + c >= Cout) break;
    float v = acc[c];
    if (relu) v = fmaxf(v, 0.f);
    y[((size_t)b * yC + yc0 + co0 + c) * V + vox(oz, oy, ox, D)] = v;
  }
}

// wT[ci][co][k] = w[co][ci][26 - k]: the weights of the transposed
// (data-gradient) convolution.
__global__ void k_conv3_wT(const __nv_bfloat16* __restrict__ w, int Cout, int Cin,
                           __nv_bfloat16* __restrict__ wT) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Cout * Cin * 27) return;
  const int k = q % 27, ci = (q / 27) % Cin, co = q / (27 * Cin);
  wT[((size_t)ci * Cout + co) * 27 + (26 - k)] = w[q];
}

// dw[co][ci][k] = sum_b sum_p dy[b][co][p] x[b][xc0 + ci][p + off(k)], and
// (ci == 0) db[co] = sum dy.  CTA per (co, ci); fixed-order reduction.
__global__ void __launch_bounds__(256)
    k_conv3_dw(const float* __restrict__ x, int xC, int xc0, int Cin,
               const float* __restrict__ dy, int dyC, int dyc0, int Cout, int D, int B,
               float* __restrict__ dw, float* __restrict__ db) {
  const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
  const size_t V = (size_t)D * D * D;
  float s[28];
#pragma unroll
  for (int k = 0; k < 28; ++k) s[k] = 0.f;
  for (size_t e = threadIdx.x; e < (size_t)B * V; e += blockDim.x) {
    const int b = (int)(e / V), p = (int)(e % V);
    const int px = p % D, py = (p / D) % D, pz = p / (D * D);
    const float g = dy[((size_t)b * dyC + dyc0 + co) * V + p];
    const float* xs = x + ((size_t)b * xC + xc0 + ci) * V;
    s[27] += g;
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const int gx = px + k % 3 - 1, gy = py + (k / 3) % 3 - 1, gz = pz + k / 9 - 1;
      const float xv = (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D)
                           ? xs[vox(gz, gy, gx, D)]
                           : 0.f;
      s[k] = fmaf(g, xv, s[k]);
    }
  }
  __shared__ float red[28][256];
#pragma unroll
  for (int k = 0; k < 28; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int k = 0; k < 28; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 27) dw[((size_t)co * Cin + ci) * 27 + threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 27 && ci == 0 && db) db[co] = red[27][0];
}

// g[b][c][p] *= (y[b][c][p] > 0) over a channel slice (the ReLU's gradient).
__global__ void k_relu_bwd(float* __restrict__ g, int gC, int gc0, const float* __restrict__ y,
                           int yC, int yc0, int C, size_t V, int B) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * V) return;
  const size_t p = q % V;
  const int c = (int)((q / V) % C), b = (int)(q / (V * C));
  if (!(y[((size_t)b * yC + yc0 + c) * V + p] > 0.f)) g[((size_t)b * gC + gc0 + c) * V + p] = 0.f;
}

// 2x average pooling of a channel slice: D -> D / 2.
__global__ void k_pool(const float* __restrict__ x, int xC, int xc0, float* __restrict__ y, int C,
                       int D, int B) {
  const int Dh = D / 2;
  const size_t Vh = (size_t)Dh * Dh * Dh;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * Vh) return;
  const int p = (int)(q % Vh), c = (int)((q / Vh) % C), b = (int)(q / (Vh * C));
  const int px = p % Dh, py = (p / Dh) % Dh, pz = p / (Dh * Dh);
  const float* xs = x + ((size_t)b * xC + xc0 + c) * ((size_t)D * D * D);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += xs[vox(2 * pz + k / 4, 2 * py + (k / 2) % 2, 2 * px + k % 2, D)];
  y[q] = 0.125f * s;
}

// Gradient of the pooling: dx[child] (+)= dy[parent] / 8 into a slice.
__global__ void k_pool_bwd(const float* __restrict__ dy, float* __restrict__ dx, int xC, int xc0,
                           int C, int D, int B, int add) {
  const size_t V = (size_t)D * D * D;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * V) return;
  const int p = (int)(q % V), c = (int)((q / V) % C), b = (int)(q / (V * C));
  const int Dh = D / 2;
  const int px = p % D, py = (p / D) % D, pz = p / (D * D);
  const float g = 0.125f * dy[((size_t)b * C + c) * ((size_t)Dh * Dh * Dh) + vox(pz / 2, py / 2, px / 2, Dh)];
  float* d = dx + ((size_t)b * xC + xc0 + c) * V + p;
  *d = add ? *d + g : g;
}

// Nearest 2x upsampling into a channel slice: D -> 2D.
__global__ void k_up(const float* __restrict__ x, int C, int D, float* __restrict__ y, int yC,
                     int yc0, int B) {
  const int D2 = 2 * D;
  const size_t V2 = (size_t)D2 * D2 * D2;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * V2) return;
  const int p = (int)(q % V2), c = (int)((q / V2) % C), b = (int)(q / (V2 * C));
  const int px = p % D2, py = (p / D2) % D2, pz = p / (D2 * D2);
  y[((size_t)b * yC + yc0 + c) * V2 + p] =
      x[((size_t)b * C + c) * ((size_t)D * D * D) + vox(pz / 2, py / 2, px / 2, D)];
}

// Gradient of the upsampling: dx[parent] = sum of the 8 children (fixed order).
__global__ void k_up_bwd(const float* __restrict__ dy, int yC, int yc0, float* __restrict__ dx,
                         int C, int D, int B) {
  const size_t V = (size_t)D * D * D;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * V) return;
  const int p = (int)(q % V), c = (int)((q / V) % C), b = (int)(q / (V * C));
  const int px = p % D, py = (p / D) % D, pz = p / (D * D);
  const int D2 = 2 * D;
  const float* g = dy + ((size_t)b * yC + yc0 + c) * ((size_t)D2 * D2 * D2);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += g[vox(2 * pz + k / 4, 2 * py + (k / 2) % 2, 2 * px + k % 2, D2)];
  dx[q] = s;
}

// out[b][p] = bias + sum_c w[c] x[b][c][p]  (1x1x1 convolution to 1 channel)
__global__ void k_conv1(const float* __restrict__ x, int C, const __nv_bfloat16* __restrict__ w,
                        const float* __restrict__ bias, float* __restrict__ out, size_t V, int B) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * V) return;
  const size_t p = q % V;
  const int b = (int)(q / V);
  float s = bias[0];
  for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(w[c]), x[((size_t)b * C + c) * V + p], s);
  out[q] = s;
}

// dx[b][c][p] = w[c] dy[b][p]
__global__ void k_conv1_dx(const float* __restrict__ dy, int C, const __nv_bfloat16* __restrict__ w,
                           float* __restrict__ dx, size_t V, int B) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * C * V) return;
  const size_t p = q % V;
  const int c = (int)((q / V) % C), b = (int)(q / (V * C));
  dx[q] = __bfloat162float(w[c]) * dy[(size_t)b * V + p];
}

// dw[c] = sum dy x[c], db = sum dy: CTA per c (c == C: the bias).
__global__ void __launch_bounds__(256)
    k_conv1_dw(const float* __restrict__ x, int C, const float* __restrict__ dy, size_t V, int B,
               float* __restrict__ dw, float* __restrict__ db) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (size_t e = threadIdx.x; e < (size_t)B * V; e += blockDim.x) {
    const size_t p = e % V;
    const int b = (int)(e / V);
    const float g = dy[e];
    s = c < C ? fmaf(g, x[((size_t)b * C + c) * V + p], s) : s + g;
  }
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (c < C)
      dw[c] = red[0];
    else
      db[0] = red[0];
  }
}

// Masked mean squared error: loss = sum m (y - t)^2 / sum m (m = input
// channel 1), dy = 2 m (y - t) / sum m.  One CTA, fixed order.
__global__ void __launch_bounds__(1024)
    k_loss(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ in,
           size_t V, int B, float* __restrict__ dy, double* __restrict__ loss) {
  double se = 0.0, sm = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)B * V; e += blockDim.x) {
    const size_t p = e % V;
    const int b = (int)(e / V);
    const double m = in[((size_t)b * 2 + 1) * V + p];
    const double d = (double)y[e] - (double)t[e];
    se += m * d * d;
    sm += m;
  }
  __shared__ double r1[1024], r2[1024];
  r1[threadIdx.x] = se;
  r2[threadIdx.x] = sm;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r1[threadIdx.x] += r1[threadIdx.x + h];
      r2[threadIdx.x] += r2[threadIdx.x + h];
    }
    __syncthreads();
  }
  const double msum = r2[0] > 0.0 ? r2[0] : 1.0;
  if (threadIdx.x == 0) *loss = r1[0] / msum;
  if (!dy) return;
  for (size_t e = threadIdx.x; e < (size_t)B * V; e += blockDim.x) {
    const size_t p = e % V;
    const int b = (int)(e / V);
    const float m = in[((size_t)b * 2 + 1) * V + p];
    dy[e] = (float)(2.0 * m * ((double)y[e] - (double)t[e]) / msum);
  }
}

// Adam on the FP32 master weights; BF16 copy for the kernels.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16* __restrict__ wb) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  w[q] = wq;
  wb[q] = __float2bfloat16(wq);
}

__global__ void k_to_bf16(const float* __restrict__ w, long long n, __nv_bfloat16* __restrict__ wb) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) wb[q] = __float2bfloat16(w[q]);
}

// Patches of pairs: input [2][32^3] = (b / s, box mask), target v / s (if
// v), s = max |b| on the box; the box interior (ext <= 32 per axis) at
// offset (32 - ext) / 2.  CTA per pair; pairs that do not fit get s = 0
// and zero patches.
__global__ void __launch_bounds__(256)
    k_patch(const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff, int P,
            const double* __restrict__ bbuf, const double* __restrict__ vbuf,
            float* __restrict__ in, float* __restrict__ tgt, double* __restrict__ scale) {
  const int p = blockIdx.x;
  const PairInfo Pi = pinfo[p];
  const bool fits = Pi.ext[0] <= UN_P && Pi.ext[1] <= UN_P && Pi.ext[2] <= UN_P;
  const double* b = bbuf + voff[p];
  __shared__ double red[256];
  double mx = 0.0;
  if (fits)
    for (int t = threadIdx.x; t < Pi.n; t += blockDim.x) mx = fmax(mx, fabs(b[t]));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  const double s = red[0];
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  if (threadIdx.x == 0) scale[p] = fits ? s : 0.0;
  float* ib = in + (size_t)p * 2 * UN_V;
  float* im = ib + UN_V;
  float* tg = tgt ? tgt + (size_t)p * UN_V : nullptr;
  const int ox = (UN_P - Pi.ext[0]) / 2, oy = (UN_P - Pi.ext[1]) / 2, oz = (UN_P - Pi.ext[2]) / 2;
  for (int q = threadIdx.x; q < UN_V; q += blockDim.x) {
    const int x = q % UN_P - ox, y = (q / UN_P) % UN_P - oy, z = q / (UN_P * UN_P) - oz;
    const bool in_box = fits && x >= 0 && x < Pi.ext[0] && y >= 0 && y < Pi.ext[1] && z >= 0 &&
                        z < Pi.ext[2];
    const int t = in_box ? (z * Pi.ext[1] + y) * Pi.ext[0] + x : 0;
    ib[q] = in_box ? (float)(b[t] * inv) : 0.f;
    im[q] = in_box ? 1.f : 0.f;
    if (tg) tg[q] = in_box ? (float)(vbuf[voff[p] + t] * inv) : 0.f;
  }
}

// x0 on each pair's box = s * prediction (0 where the pair did not fit).
__global__ void k_unpatch(const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff,
                          int p0, int np, const float* __restrict__ pred,
                          const double* __restrict__ scale, double* __restrict__ x) {
  const int p = p0 + blockIdx.x;
  if (blockIdx.x >= np) return;
  const PairInfo Pi = pinfo[p];
  const double s = scale[p];
  const int ox = (UN_P - Pi.ext[0]) / 2, oy = (UN_P - Pi.ext[1]) / 2, oz = (UN_P - Pi.ext[2]) / 2;
  const float* pr = pred + (size_t)blockIdx.x * UN_V;
  for (int t = threadIdx.x; t < Pi.n; t += blockDim.x) {
    if (s == 0.0) {
      x[voff[p] + t] = 0.0;
      continue;
    }
    const int xx = t % Pi.ext[0], yy = (t / Pi.ext[0]) % Pi.ext[1], zz = t / (Pi.ext[0] * Pi.ext[1]);
    x[voff[p] + t] = s * (double)pr[vox(zz + oz, yy + oy, xx + ox, UN_P)];
  }
}

}  // namespace
}  // namespace sea

// ---------------------------------------------------------------------------
// Model object (host side)
// ---------------------------------------------------------------------------
struct UnLayer {
  int cin, cout, k;           // k = 3 (3x3x3) or 1
  long long w_off, b_off;     // offsets in the parameter array
};

struct sea_unet {
  int width = 16, device = 0, bmax = 32;
  cudaStream_t stream = nullptr;
  std::vector<UnLayer> L;
  long long nparam = 0;
  float *master = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  __nv_bfloat16 *wb = nullptr, *wT = nullptr;
  int adam_t = 0;
  // activations and gradients for a batch of up to bmax patches
  float *e1a = nullptr, *cat1 = nullptr, *p1 = nullptr, *e2a = nullptr, *cat2 = nullptr,
        *p2 = nullptr, *b4 = nullptr, *b5 = nullptr, *d2a = nullptr, *d2b = nullptr,
        *d1a = nullptr, *d1b = nullptr, *out = nullptr;
  float *g32a = nullptr, *g32b = nullptr, *g16a = nullptr, *g16b = nullptr, *g8a = nullptr,
        *g8b = nullptr, *gcat1 = nullptr, *gcat2 = nullptr, *gout = nullptr;
  double* dloss = nullptr;
  // training set
  float *tin = nullptr, *ttg = nullptr;
  long long ns = 0, cap = 0;
  // inference scratch for contexts
  float* pin = nullptr;
  double* pscale = nullptr;
  long long pcap = 0;
  char err[256] = {0};
};

namespace {

bool alloc(void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; }

sea_status un_fail(sea_unet* u, sea_status st, const char* msg) {
  if (u) snprintf(u->err, sizeof(u->err), "%s", msg);
  return st;
}

unsigned grid1(size_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

void conv3(sea_unet* u, const float* x, int xC, int xc0, int l, float* y, int yC, int yc0, int D,
           int B, int relu) {
  const UnLayer& a = u->L[l];
  const int tiles = ((D + 7) / 8) * ((D + 7) / 8) * ((D + 3) / 4);
  sea::k_conv3<<<dim3(tiles, (a.cout + CV_CO - 1) / CV_CO, B), 256, 0, u->stream>>>(
      x, xC, xc0, a.cin, u->wb + a.w_off, u->master + a.b_off, y, yC, yc0, a.cout, D, relu);
}

// dx (slice of a tensor with xC channels) = transposed convolution of dy
void conv3_dx(sea_unet* u, int l, const float* dy, int dyC, float* dx, int xC, int xc0, int D,
              int B) {
  const UnLayer& a = u->L[l];
  sea::k_conv3_wT<<<grid1((size_t)a.cout * a.cin * 27), 256, 0, u->stream>>>(u->wb + a.w_off, a.cout,
                                                                             a.cin, u->wT);
  const int tiles = ((D + 7) / 8) * ((D + 7) / 8) * ((D + 3) / 4);
  sea::k_conv3<<<dim3(tiles, (a.cin + CV_CO - 1) / CV_CO, B), 256, 0, u->stream>>>(
      dy, dyC, 0, a.cout, u->wT, nullptr, dx, xC, xc0, a.cin, D, 0);
}

void conv3_dw(sea_unet* u, int l, const float* x, int xC, int xc0, const float* dy, int dyC, int D,
              int B) {
  const UnLayer& a = u->L[l];
  sea::k_conv3_dw<<<a.cout * a.cin, 256, 0, u->stream>>>(x, xC, xc0, a.cin, dy, dyC, 0, a.cout, D,
                                                          B, u->grad + a.w_off, u->grad + a.b_off);
}

void relu_bwd(sea_unet* u, float* g, int gC, int gc0, const float* y, int yC, int yc0, int C, int D,
              int B) {
  const size_t V = (size_t)D * D * D;
  sea::k_relu_bwd<<<grid1((size_t)B * C * V), 256, 0, u->stream>>>(g, gC, gc0, y, yC, yc0, C, V, B);
}

// Forward pass on B patches at `in` ([B][2][32^3]); output in u->out.
void forward(sea_unet* u, const float* in, int B) {
  const int c = u->width;
  const size_t V32 = UN_V, V16 = V32 / 8;
  conv3(u, in, 2, 0, 0, u->e1a, c, 0, 32, B, 1);
  conv3(u, u->e1a, c, 0, 1, u->cat1, 3 * c, 2 * c, 32, B, 1);  // skip 1 into cat1[2c..3c)
  sea::k_pool<<<grid1((size_t)B * c * V16), 256, 0, u->stream>>>(u->cat1, 3 * c, 2 * c, u->p1, c, 32, B);
  conv3(u, u->p1, c, 0, 2, u->e2a, 2 * c, 0, 16, B, 1);
  conv3(u, u->e2a, 2 * c, 0, 3, u->cat2, 6 * c, 4 * c, 16, B, 1);  // skip 2 into cat2[4c..6c)
  sea::k_pool<<<grid1((size_t)B * 2 * c * (V16 / 8)), 256, 0, u->stream>>>(u->cat2, 6 * c, 4 * c,
                                                                           u->p2, 2 * c, 16, B);
  conv3(u, u->p2, 2 * c, 0, 4, u->b4, 4 * c, 0, 8, B, 1);
  conv3(u, u->b4, 4 * c, 0, 5, u->b5, 4 * c, 0, 8, B, 1);
  sea::k_up<<<grid1((size_t)B * 4 * c * V16), 256, 0, u->stream>>>(u->b5, 4 * c, 8, u->cat2, 6 * c, 0, B);
  conv3(u, u->cat2, 6 * c, 0, 6, u->d2a, 2 * c, 0, 16, B, 1);
  conv3(u, u->d2a, 2 * c, 0, 7, u->d2b, 2 * c, 0, 16, B, 1);
  sea::k_up<<<grid1((size_t)B * 2 * c * V32), 256, 0, u->stream>>>(u->d2b, 2 * c, 16, u->cat1, 3 * c, 0, B);
  conv3(u, u->cat1, 3 * c, 0, 8, u->d1a, c, 0, 32, B, 1);
  conv3(u, u->d1a, c, 0, 9, u->d1b, c, 0, 32, B, 1);
  const UnLayer& o = u->L[10];
  sea::k_conv1<<<grid1((size_t)B * V32), 256, 0, u->stream>>>(u->d1b, c, u->wb + o.w_off,
                                                              u->master + o.b_off, u->out, V32, B);
}

// Loss and gradients (u->grad) for B patches; forward() must have run on `in`.
void backward(sea_unet* u, const float* in, const float* tgt, int B) {
  const int c = u->width;
  const size_t V32 = UN_V, V16 = V32 / 8, V8 = V16 / 8;
  sea::k_loss<<<1, 1024, 0, u->stream>>>(u->out, tgt, in, V32, B, u->gout, u->dloss);
  const UnLayer& o = u->L[10];
  sea::k_conv1_dw<<<c + 1, 256, 0, u->stream>>>(u->d1b, c, u->gout, V32, B, u->grad + o.w_off,
                                                u->grad + o.b_off);
  sea::k_conv1_dx<<<grid1((size_t)B * c * V32), 256, 0, u->stream>>>(u->gout, c, u->wb + o.w_off,
                                                                     u->g32a, V32, B);
  // d1b = relu(conv9(d1a))
  relu_bwd(u, u->g32a, c, 0, u->d1b, c, 0, c, 32, B);
  conv3_dw(u, 9, u->d1a, c, 0, u->g32a, c, 32, B);
  conv3_dx(u, 9, u->g32a, c, u->g32b, c, 0, 32, B);
  // d1a = relu(conv8(cat1))
  relu_bwd(u, u->g32b, c, 0, u->d1a, c, 0, c, 32, B);
  conv3_dw(u, 8, u->cat1, 3 * c, 0, u->g32b, c, 32, B);
  conv3_dx(u, 8, u->g32b, c, u->gcat1, 3 * c, 0, 32, B);
  // cat1[0..2c) = up(d2b)
  sea::k_up_bwd<<<grid1((size_t)B * 2 * c * V16), 256, 0, u->stream>>>(u->gcat1, 3 * c, 0, u->g16a,
                                                                       2 * c, 16, B);
  // d2b = relu(conv7(d2a))
  relu_bwd(u, u->g16a, 2 * c, 0, u->d2b, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 7, u->d2a, 2 * c, 0, u->g16a, 2 * c, 16, B);
  conv3_dx(u, 7, u->g16a, 2 * c, u->g16b, 2 * c, 0, 16, B);
  // d2a = relu(conv6(cat2))
  relu_bwd(u, u->g16b, 2 * c, 0, u->d2a, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 6, u->cat2, 6 * c, 0, u->g16b, 2 * c, 16, B);
  conv3_dx(u, 6, u->g16b, 2 * c, u->gcat2, 6 * c, 0, 16, B);
  // cat2[0..4c) = up(b5)
  sea::k_up_bwd<<<grid1((size_t)B * 4 * c * V8), 256, 0, u->stream>>>(u->gcat2, 6 * c, 0, u->g8a,
                                                                      4 * c, 8, B);
  // b5 = relu(conv5(b4)), b4 = relu(conv4(p2))
  relu_bwd(u, u->g8a, 4 * c, 0, u->b5, 4 * c, 0, 4 * c, 8, B);
  conv3_dw(u, 5, u->b4, 4 * c, 0, u->g8a, 4 * c, 8, B);
  conv3_dx(u, 5, u->g8a, 4 * c, u->g8b, 4 * c, 0, 8, B);
  relu_bwd(u, u->g8b, 4 * c, 0, u->b4, 4 * c, 0, 4 * c, 8, B);
  conv3_dw(u, 4, u->p2, 2 * c, 0, u->g8b, 4 * c, 8, B);
  conv3_dx(u, 4, u->g8b, 4 * c, u->g8a, 2 * c, 0, 8, B);  // d p2
  // p2 = pool(cat2[4c..6c)): add into the skip-2 gradient slice of gcat2
  sea::k_pool_bwd<<<grid1((size_t)B * 2 * c * V16), 256, 0, u->stream>>>(u->g8a, u->gcat2, 6 * c,
                                                                        4 * c, 2 * c, 16, B, 1);
  // skip 2 = relu(conv3(e2a))
  relu_bwd(u, u->gcat2, 6 * c, 4 * c, u->cat2, 6 * c, 4 * c, 2 * c, 16, B);
  {
    const UnLayer& a = u->L[3];
    sea::k_conv3_dw<<<a.cout * a.cin, 256, 0, u->stream>>>(u->e2a, 2 * c, 0, a.cin, u->gcat2, 6 * c,
                                                            4 * c, a.cout, 16, B, u->grad + a.w_off,
                                                            u->grad + a.b_off);
    sea::k_conv3_wT<<<grid1((size_t)a.cout * a.cin * 27), 256, 0, u->stream>>>(u->wb + a.w_off,
                                                                               a.cout, a.cin, u->wT);
    const int tiles = 2 * 2 * 4;
    sea::k_conv3<<<dim3(tiles, (a.cin + CV_CO - 1) / CV_CO, B), 256, 0, u->stream>>>(
        u->gcat2, 6 * c, 4 * c, a.cout, u->wT, nullptr, u->g16a, 2 * c, 0, a.cin, 16, 0);
  }
  // e2a = relu(conv2(p1))
  relu_bwd(u, u->g16a, 2 * c, 0, u->e2a, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 2, u->p1, c, 0, u->g16a, 2 * c, 16, B);
  conv3_dx(u, 2, u->g16a, 2 * c, u->g16b, c, 0, 16, B);  // d p1
  // p1 = pool(cat1[2c..3c)): add into the skip-1 gradient slice of gcat1
  sea::k_pool_bwd<<<grid1((size_t)B * c * V32), 256, 0, u->stream>>>(u->g16b, u->gcat1, 3 * c, 2 * c,
                                                                     c, 32, B, 1);
  // skip 1 = relu(conv1(e1a))
  relu_bwd(u, u->gcat1, 3 * c, 2 * c, u->cat1, 3 * c, 2 * c, c, 32, B);
  {
    const UnLayer& a = u->L[1];
    sea::k_conv3_dw<<<a.cout * a.cin, 256, 0, u->stream>>>(u->e1a, c, 0, a.cin, u->gcat1, 3 * c,
                                                            2 * c, a.cout, 32, B, u->grad + a.w_off,
                                                            u->grad + a.b_off);
    sea::k_conv3_wT<<<grid1((size_t)a.cout * a.cin * 27), 256, 0, u->stream>>>(u->wb + a.w_off,
                                                                               a.cout, a.cin, u->wT);
    const int tiles = 4 * 4 * 8;
    sea::k_conv3<<<dim3(tiles, (a.cin + CV_CO - 1) / CV_CO, B), 256, 0, u->stream>>>(
        u->gcat1, 3 * c, 2 * c, a.cout, u->wT, nullptr, u->g32a, c, 0, a.cin, 32, 0);
  }
  // e1a = relu(conv0(in))
  relu_bwd(u, u->g32a, c, 0, u->e1a, c, 0, c, 32, B);
  conv3_dw(u, 0, in, 2, 0, u->g32a, c, 32, B);
}

}  // namespace

extern "C" {

long long sea_unet_num_weights(const sea_unet* u) { return u ? u->nparam : 0; }

const char* sea_unet_last_error(const sea_unet* u) {
  if (!u) return "NULL model";
  return u->err[0] ? u->err : "no error";
}

void sea_unet_destroy(sea_unet* u) {
  if (!u) return;
  cudaStreamSynchronize(u->stream);
  float* fs[] = {u->master, u->grad, u->am, u->av, u->e1a, u->cat1, u->p1, u->e2a, u->cat2,
                 u->p2, u->b4, u->b5, u->d2a, u->d2b, u->d1a, u->d1b, u->out, u->g32a, u->g32b,
                 u->g16a, u->g16b, u->g8a, u->g8b, u->gcat1, u->gcat2, u->gout, u->tin, u->ttg,
                 u->pin};
  for (float* p : fs)
    if (p) cudaFree(p);
  if (u->wb) cudaFree(u->wb);
  if (u->wT) cudaFree(u->wT);
  if (u->dloss) cudaFree(u->dloss);
  if (u->pscale) cudaFree(u->pscale);
  delete u;
}

sea_status sea_unet_create(int width, int seed, void* cuda_stream, sea_unet** out) {
  if (!out || width < 1 || width > 64) return SEA_ERR_ARG;
  *out = nullptr;
  sea_unet* u = new (std::nothrow) sea_unet();
  if (!u) return SEA_ERR_OOM;
  u->width = width;
  u->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&u->device) != cudaSuccess) {
    delete u;
    return SEA_ERR_CUDA;
  }
  const int c = width;
  const int dims[11][3] = {{2, c, 3},         {c, c, 3},         {c, 2 * c, 3},     {2 * c, 2 * c, 3},
                           {2 * c, 4 * c, 3}, {4 * c, 4 * c, 3}, {6 * c, 2 * c, 3}, {2 * c, 2 * c, 3},
                           {3 * c, c, 3},     {c, c, 3},         {c, 1, 1}};
  long long off = 0, maxw = 0;
  for (auto& d : dims) {
    UnLayer l;
    l.cin = d[0];
    l.cout = d[1];
    l.k = d[2];
    const long long nw = (long long)l.cout * l.cin * (l.k == 3 ? 27 : 1);
    l.w_off = off;
    off += nw;
    l.b_off = off;
    off += l.cout;
    maxw = std::max(maxw, nw);
    u->L.push_back(l);
  }
  u->nparam = off;
  // He-normal weights, zero biases (seeded)
  std::vector<float> h(off, 0.f);
  std::mt19937_64 gen((unsigned long long)seed * 0x9E3779B97F4A7C15ULL + 12345ULL);
  for (const UnLayer& l : u->L) {
    const double fan_in = (double)l.cin * (l.k == 3 ? 27 : 1);
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan_in));
    for (long long q = 0; q < (long long)l.cout * l.cin * (l.k == 3 ? 27 : 1); ++q)
      h[l.w_off + q] = (float)nd(gen);
  }
  const size_t B = u->bmax, V32 = UN_V, V16 = V32 / 8, V8 = V16 / 8;
  bool ok = alloc((void**)&u->master, off * 4) && alloc((void**)&u->grad, off * 4) &&
            alloc((void**)&u->am, off * 4) && alloc((void**)&u->av, off * 4) &&
            alloc((void**)&u->wb, off * 2) && alloc((void**)&u->wT, maxw * 2) &&
            alloc((void**)&u->e1a, B * c * V32 * 4) && alloc((void**)&u->cat1, B * 3 * c * V32 * 4) &&
            alloc((void**)&u->p1, B * c * V16 * 4) && alloc((void**)&u->e2a, B * 2 * c * V16 * 4) &&
            alloc((void**)&u->cat2, B * 6 * c * V16 * 4) && alloc((void**)&u->p2, B * 2 * c * V8 * 4) &&
            alloc((void**)&u->b4, B * 4 * c * V8 * 4) && alloc((void**)&u->b5, B * 4 * c * V8 * 4) &&
            alloc((void**)&u->d2a, B * 2 * c * V16 * 4) && alloc((void**)&u->d2b, B * 2 * c * V16 * 4) &&
            alloc((void**)&u->d1a, B * c * V32 * 4) && alloc((void**)&u->d1b, B * c * V32 * 4) &&
            alloc((void**)&u->out, B * V32 * 4) && alloc((void**)&u->g32a, B * c * V32 * 4) &&
            alloc((void**)&u->g32b, B * c * V32 * 4) && alloc((void**)&u->g16a, B * 2 * c * V16 * 4) &&
            alloc((void**)&u->g16b, B * 2 * c * V16 * 4) && alloc((void**)&u->g8a, B * 4 * c * V8 * 4) &&
            alloc((void**)&u->g8b, B * 4 * c * V8 * 4) && alloc((void**)&u->gcat1, B * 3 * c * V32 * 4) &&
            alloc((void**)&u->gcat2, B * 6 * c * V16 * 4) && alloc((void**)&u->gout, B * V32 * 4) &&
            alloc((void**)&u->dloss, 8);
  if (!ok) {
    sea_unet_destroy(u);
    return SEA_ERR_OOM;
  }
  if (cudaMemcpyAsync(u->master, h.data(), off * 4, cudaMemcpyHostToDevice, u->stream) != cudaSuccess ||
      cudaMemsetAsync(u->am, 0, off * 4, u->stream) != cudaSuccess ||
      cudaMemsetAsync(u->av, 0, off * 4, u->stream) != cudaSuccess) {
    sea_unet_destroy(u);
    return SEA_ERR_CUDA;
  }
  sea::k_to_bf16<<<grid1(off), 256, 0, u->stream>>>(u->master, off, u->wb);
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) {
    sea_unet_destroy(u);
    return SEA_ERR_CUDA;
  }
  *out = u;
  return SEA_OK;
}

sea_status sea_unet_weights(sea_unet* u, float* w, int set) {
  if (!u || !w) return SEA_ERR_ARG;
  const size_t bytes = (size_t)u->nparam * 4;
  cudaError_t e;
  if (set) {
    e = cudaMemcpyAsync(u->master, w, bytes, cudaMemcpyHostToDevice, u->stream);
    if (e == cudaSuccess) {
      sea::k_to_bf16<<<grid1(u->nparam), 256, 0, u->stream>>>(u->master, u->nparam, u->wb);
      e = cudaGetLastError();
    }
  } else {
    e = cudaMemcpyAsync(w, u->master, bytes, cudaMemcpyDeviceToHost, u->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  return e == cudaSuccess ? SEA_OK : un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
}

sea_status sea_unet_forward(sea_unet* u, const float* in, int B, float* out, int on_device) {
  if (!u || !in || !out || B < 1) return SEA_ERR_ARG;
  for (int b0 = 0; b0 < B; b0 += u->bmax) {
    const int nb = std::min(u->bmax, B - b0);
    const float* src = in + (size_t)b0 * 2 * UN_V;
    if (!on_device) {
      if (cudaMemcpyAsync(u->gcat1, src, (size_t)nb * 2 * UN_V * 4, cudaMemcpyHostToDevice,
                          u->stream) != cudaSuccess)
        return un_fail(u, SEA_ERR_CUDA, "copy input");
      src = u->gcat1;  // scratch large enough (3c >= 2 channels)
    }
    forward(u, src, nb);
    if (cudaMemcpyAsync(out + (size_t)b0 * UN_V, u->out, (size_t)nb * UN_V * 4,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        u->stream) != cudaSuccess)
      return un_fail(u, SEA_ERR_CUDA, "copy output");
  }
  const cudaError_t e = cudaStreamSynchronize(u->stream);
  return e == cudaSuccess ? SEA_OK : un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
}

sea_status sea_unet_loss_grad(sea_unet* u, const float* in, const float* target, int B,
                              double* loss, float* grad, int on_device) {
  if (!u || !in || !target || B < 1 || B > u->bmax) return SEA_ERR_ARG;
  float* din = u->tin;
  float* dtg = u->ttg;
  const float* src_in = in;
  const float* src_tg = target;
  if (!on_device) {
    // staging in the training buffers' space would disturb them: use scratch
    if (!u->pin && !alloc((void**)&u->pin, (size_t)u->bmax * 3 * UN_V * 4))
      return un_fail(u, SEA_ERR_OOM, "staging");
    din = u->pin;
    dtg = u->pin + (size_t)u->bmax * 2 * UN_V;
    if (cudaMemcpyAsync(din, in, (size_t)B * 2 * UN_V * 4, cudaMemcpyHostToDevice, u->stream) != cudaSuccess ||
        cudaMemcpyAsync(dtg, target, (size_t)B * UN_V * 4, cudaMemcpyHostToDevice, u->stream) != cudaSuccess)
      return un_fail(u, SEA_ERR_CUDA, "copy input");
    src_in = din;
    src_tg = dtg;
  }
  cudaMemsetAsync(u->gcat1, 0, (size_t)B * 3 * u->width * UN_V * 4, u->stream);
  cudaMemsetAsync(u->gcat2, 0, (size_t)B * 6 * u->width * (UN_V / 8) * 4, u->stream);
  forward(u, src_in, B);
  backward(u, src_in, src_tg, B);
  double l = 0.0;
  cudaMemcpyAsync(&l, u->dloss, 8, cudaMemcpyDeviceToHost, u->stream);
  if (grad) cudaMemcpyAsync(grad, u->grad, (size_t)u->nparam * 4, cudaMemcpyDeviceToHost, u->stream);
  const cudaError_t e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) return un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
  if (loss) *loss = l;
  return SEA_OK;
}

sea_status sea_unet_collect(sea_unet* u, sea_ctx* c) {
  if (!u || !c) return SEA_ERR_ARG;
  if (!c->have_vxx || c->P == 0) return un_fail(u, SEA_ERR_STATE, "no sea_apply_vxx result");
  const long long need = u->ns + c->P;
  if (need > u->cap) {
    const long long cap = std::max(need, u->cap * 2);
    float *ni = nullptr, *nt = nullptr;
    if (!alloc((void**)&ni, (size_t)cap * 2 * UN_V * 4) || !alloc((void**)&nt, (size_t)cap * UN_V * 4)) {
      if (ni) cudaFree(ni);
      return un_fail(u, SEA_ERR_OOM, "training set");
    }
    if (u->ns) {
      cudaMemcpyAsync(ni, u->tin, (size_t)u->ns * 2 * UN_V * 4, cudaMemcpyDeviceToDevice, u->stream);
      cudaMemcpyAsync(nt, u->ttg, (size_t)u->ns * UN_V * 4, cudaMemcpyDeviceToDevice, u->stream);
    }
    cudaStreamSynchronize(u->stream);
    if (u->tin) cudaFree(u->tin);
    if (u->ttg) cudaFree(u->ttg);
    u->tin = ni;
    u->ttg = nt;
    u->cap = cap;
  }
  double* scale = nullptr;
  if (!alloc((void**)&scale, (size_t)c->P * 8)) return un_fail(u, SEA_ERR_OOM, "scales");
  cudaStreamSynchronize(c->stream);
  sea::k_patch<<<c->P, 256, 0, u->stream>>>((const PairInfo*)c->pinfo.p, (const long long*)c->voff.p,
                                            c->P, (const double*)c->bbuf.p, (const double*)c->vbuf.p,
                                            u->tin + (size_t)u->ns * 2 * UN_V,
                                            u->ttg + (size_t)u->ns * UN_V, scale);
  cudaError_t e = cudaStreamSynchronize(u->stream);
  cudaFree(scale);
  if (e != cudaSuccess) return un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
  u->ns += c->P;
  return SEA_OK;
}

long long sea_unet_num_samples(const sea_unet* u) { return u ? u->ns : 0; }

sea_status sea_unet_train(sea_unet* u, int steps, int batch, double lr, int seed,
                          double* last_loss) {
  if (!u || steps < 0 || batch < 1 || batch > u->bmax || !(lr > 0.0)) return SEA_ERR_ARG;
  if (u->ns < batch) return un_fail(u, SEA_ERR_STATE, "fewer collected samples than the batch");
  if (!u->pin && !alloc((void**)&u->pin, (size_t)u->bmax * 3 * UN_V * 4))
    return un_fail(u, SEA_ERR_OOM, "batch buffer");
  float* bin = u->pin;
  float* btg = u->pin + (size_t)u->bmax * 2 * UN_V;
  std::mt19937_64 gen((unsigned long long)seed * 0x2545F4914F6CDD1DULL + 99ULL);
  std::uniform_int_distribution<long long> pick(0, u->ns - 1);
  double l = 0.0;
  for (int s = 0; s < steps; ++s) {
    for (int b = 0; b < batch; ++b) {
      const long long k = pick(gen);
      cudaMemcpyAsync(bin + (size_t)b * 2 * UN_V, u->tin + (size_t)k * 2 * UN_V, 2 * UN_V * 4,
                      cudaMemcpyDeviceToDevice, u->stream);
      cudaMemcpyAsync(btg + (size_t)b * UN_V, u->ttg + (size_t)k * UN_V, UN_V * 4,
                      cudaMemcpyDeviceToDevice, u->stream);
    }
    cudaMemsetAsync(u->gcat1, 0, (size_t)batch * 3 * u->width * UN_V * 4, u->stream);
    cudaMemsetAsync(u->gcat2, 0, (size_t)batch * 6 * u->width * (UN_V / 8) * 4, u->stream);
    forward(u, bin, batch);
    backward(u, bin, btg, batch);
    ++u->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u->adam_t), c2 = 1.f - std::pow(b2, (float)u->adam_t);
    sea::k_adam<<<grid1(u->nparam), 256, 0, u->stream>>>(u->master, u->grad, u->am, u->av, u->nparam,
                                                        (float)lr, b1, b2, 1e-8f, c1, c2, u->wb);
  }
  if (steps > 0) cudaMemcpyAsync(&l, u->dloss, 8, cudaMemcpyDeviceToHost, u->stream);
  const cudaError_t e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) return un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
  if (last_loss) *last_loss = l;
  return SEA_OK;
}

sea_status sea_unet_attach(sea_ctx* c, sea_unet* u) {
  if (!c) return SEA_ERR_ARG;
  c->unet = u;
  return SEA_OK;
}

}  // extern "C"

namespace sea {

// Warm start of the context's CG: x0 = s * U-Net(b / s, mask) on every pair
// whose box fits the patch (0 elsewhere), written into the solution buffer,
// then 4 damped Jacobi sweeps (omega = 2/3) on it.
cudaError_t launch_warm_start(sea_ctx* c) {
  sea_unet* u = c->unet;
  if (!u || c->P == 0) return cudaSuccess;
  const int B = u->bmax;
  if (u->pcap < c->P) {
    if (u->pscale) cudaFree(u->pscale);
    u->pscale = nullptr;
    u->pcap = 0;
    if (!alloc((void**)&u->pscale, (size_t)c->P * 8)) return cudaErrorMemoryAllocation;
    u->pcap = c->P;
  }
  if (!u->pin && !alloc((void**)&u->pin, (size_t)u->bmax * 3 * UN_V * 4))
    return cudaErrorMemoryAllocation;
  // The model runs on the context's stream here.
  cudaStream_t saved = u->stream;
  u->stream = c->stream;
  for (int p0 = 0; p0 < c->P; p0 += B) {
    const int np = std::min(B, c->P - p0);
    k_patch<<<np, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p + p0,
                                       (const long long*)c->voff.p + p0, np,
                                       (const double*)c->bbuf.p, nullptr, u->pin, nullptr,
                                       u->pscale + p0);
    forward(u, u->pin, np);
    k_unpatch<<<np, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p, (const long long*)c->voff.p, p0,
                                         np, u->out, u->pscale, (double*)c->vbuf.p);
    c->launches += 2 + 15;
  }
  u->stream = saved;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // smooth the guesses' high-frequency error before the CG
  return launch_smooth(c, 4, 2.0 / 3.0);
}

}  // namespace sea
