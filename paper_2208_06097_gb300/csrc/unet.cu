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
// for the optimizer), activations FP32.  The 3x3x3 convolutions of the
// forward pass and their data gradients run on the tensor cores (tcgen05,
// kind::f16, BF16 operands, FP32 accumulation in tensor memory) as an
// implicit GEMM; each FP32 activation enters as the exact sum of three BF16
// terms, so the products are those of the FP32 values.  The weight
// gradients run on the tensor cores too (two BF16 terms per value).  Training: masked
// mean squared error against the CG solution, Adam.  All reductions run in a
// fixed order (no floating-point atomics), so training is deterministic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "sea_internal.cuh"
#include "tcgen05.cuh"

#define UN_P 32                         // patch edge
#define UN_V (UN_P * UN_P * UN_P)       // patch points

namespace sea {
namespace {

__device__ __forceinline__ int vox(int z, int y, int x, int D) { return (z * D + y) * D + x; }

// ---------------------------------------------------------------------------
// 3x3x3 convolution on the tensor cores (implicit GEMM).
//
//   y[b][yc0 + co][p] = act(bias[co] + sum_ci sum_k W[co][ci][k] x[b][xc0 + ci][p + off(k)])
//
// CTA = one tile of 8 (x) x 16 (y) x 1 (z) output points of one batch
// element (M = 128 rows: row m = y 8 + x) and up to 128 output channels
// (N).  The input is staged per chunk of 16 channels as the haloed box
// 10 x 18 x 3 around the tile, point after point (row r = (hz 18 + hy) 10 +
// hx, 16 bytes = 8 channels per row, one plane per channel octet), so that
// the A operand of offset k = (kz, ky, kx) is the same layout shifted by
// (kz 180 + ky 10 + kx) rows: core matrices of 8 x-consecutive points
// (rows 16 B apart), the next y at 160 B, the next octet one plane further.
// No im2col copy is made; each chunk costs 27 offsets x 3 terms MMAs (M =
// 128, K = 16, N = the padded channel count) into one FP32 accumulator in
// tensor memory.  Each FP32 value v enters as h + m + l, three BF16 terms
// (h = bf16(v), m = bf16(v - h), l = bf16(v - h - m): exact, every
// difference is representable), so every product is exact and only the FP32
// accumulation rounds.  Weights come prepared per chunk (k_conv_wprep) in
// the B layout [k][octet][8-row group of channels][8 x 8].  Points outside
// the volume read zeros; rows beyond D (the 8^3 level uses half a tile) are
// not stored.  The wait for the MMAs is bounded (SEA_FLAG_WAIT).
// ---------------------------------------------------------------------------
#define CT_THREADS 256
#define CT_HX 10
#define CT_HY 18
#define CT_ROWS (CT_HX * CT_HY * 3)             // 540 haloed points
#define CT_PLANE (CT_ROWS * 16)                 // one channel octet of the box, bytes
#define CT_XBYTES (3 * 2 * CT_PLANE)            // three terms x two octets
#define CT_NBLK 128                             // output channels per CTA at most

struct ConvTc {
  const float* x;
  int xC, xc0, Cin;
  const __nv_bfloat16* wp;  // prepared weights of the layer (k_conv_wprep)
  int npad;                 // output channels padded to 16 (the prepared layout's N)
  const float* bias;        // or null
  float* y;
  int yC, yc0, Cout;
  int D, relu;
  unsigned* status;
};

// Prepared weights: wp[chunk][k][o][g][r][c] = W'[co = 8 g + r][ci = 16 chunk
// + 8 o + c][k] (zero beyond Cout', Cin'), with W' = W (forward) or, for
// the data gradient (transpose = 1), W'[co'][ci'][k] = W[ci'][co'][26 - k]
// (Cout' = cin, Cin' = cout of the layer).  w: [cout][cin][27] BF16.
__global__ void k_conv_wprep(const __nv_bfloat16* __restrict__ w, int cout, int cin, int transpose,
                             int npad, __nv_bfloat16* __restrict__ wp) {
  const int Co = transpose ? cin : cout, Ci = transpose ? cout : cin;
  const int ng = npad / 8, nch = (Ci + 15) / 16;
  const long long total = (long long)nch * 27 * 2 * ng * 64;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int c = (int)(q & 7), r = (int)((q >> 3) & 7);
  long long t = q >> 6;
  const int g = (int)(t % ng);
  t /= ng;
  const int o = (int)(t & 1);
  t >>= 1;
  const int k = (int)(t % 27), ch = (int)(t / 27);
  const int co = 8 * g + r, ci = 16 * ch + 8 * o + c;
  __nv_bfloat16 v = __float2bfloat16(0.f);
  if (co < Co && ci < Ci)
    v = transpose ? w[((size_t)ci * cin + co) * 27 + (26 - k)] : w[((size_t)co * cin + ci) * 27 + k];
  wp[q] = v;
}

__device__ __forceinline__ void split3_bf16(float v0, float v1, uint32_t& h, uint32_t& m,
                                            uint32_t& l) {
  const __nv_bfloat162 H = __floats2bfloat162_rn(v0, v1);
  const float r0 = v0 - __low2float(H), r1 = v1 - __high2float(H);
  const __nv_bfloat162 Mm = __floats2bfloat162_rn(r0, r1);
  const __nv_bfloat162 L = __floats2bfloat162_rn(r0 - __low2float(Mm), r1 - __high2float(Mm));
  h = *reinterpret_cast<const uint32_t*>(&H);
  m = *reinterpret_cast<const uint32_t*>(&Mm);
  l = *reinterpret_cast<const uint32_t*>(&L);
}

__global__ void __launch_bounds__(CT_THREADS) k_conv3_tc(ConvTc P) {
  extern __shared__ unsigned char ct_raw[];
  unsigned char* sX = ct_raw + ((128 - (smem_addr(ct_raw) & 127)) & 127);
  unsigned char* sW = sX + CT_XBYTES;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tbase;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = P.D, ntx = D / 8, nty = (D + 15) / 16;
  int t = blockIdx.x;
  const int x0 = (t % ntx) * 8;
  t /= ntx;
  const int y0 = (t % nty) * 16, z0 = t / nty;
  const int b = blockIdx.y, n0 = blockIdx.z * CT_NBLK;
  const int nb = min(CT_NBLK, P.npad - n0);  // this CTA's N (a multiple of 16)
  const int ngb = nb / 8, ng = P.npad / 8;
  const uint32_t ncols = nb <= 32 ? 32u : (nb <= 64 ? 64u : 128u);
  const uint32_t mb = smem_addr(&bar);
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (tid == 0) {
    mbar_init(mb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const size_t V = (size_t)D * D * D;
  const int nch = (P.Cin + 15) / 16;
  const uint32_t idesc = idesc_kf16(nb, 128, true);
  const uint32_t ax = smem_addr(sX), aw = smem_addr(sW);
  // Thread 0 issues the MMAs and alone waits for their completion (phase:
  // parity of the next completion); the block learns the outcome through
  // s_fail after a barrier.
  uint32_t phase = 0;
  bool pending = false;  // MMAs committed and not yet waited for (uniform)
  for (int ch = 0; ch < nch; ++ch) {
    if (pending) {  // the previous chunk's MMAs read the buffers about to be replaced
      if (tid == 0) {
        if (mbar_wait(mb, phase))
          phase ^= 1;
        else
          s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      pending = false;
    }
    // the haloed input of channels 16 ch .. 16 ch + 15, three BF16 terms
    for (int it = tid; it < 2 * CT_ROWS; it += CT_THREADS) {
      const int o = it / CT_ROWS, row = it - o * CT_ROWS;
      const int hx = row % CT_HX, hy = (row / CT_HX) % CT_HY, hz = row / (CT_HX * CT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool in = gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D;
      const size_t pofs = in ? ((size_t)gz * D + gy) * D + gx : 0;
      uint32_t w[3][4];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const int ci = 16 * ch + 8 * o + 2 * c2;
        const float v0 = (in && ci < P.Cin) ? P.x[((size_t)b * P.xC + P.xc0 + ci) * V + pofs] : 0.f;
        const float v1 =
            (in && ci + 1 < P.Cin) ? P.x[((size_t)b * P.xC + P.xc0 + ci + 1) * V + pofs] : 0.f;
        split3_bf16(v0, v1, w[0][c2], w[1][c2], w[2][c2]);
      }
#pragma unroll
      for (int t3 = 0; t3 < 3; ++t3)
        *reinterpret_cast<uint4*>(sX + (t3 * 2 + o) * CT_PLANE + row * 16) =
            make_uint4(w[t3][0], w[t3][1], w[t3][2], w[t3][3]);
    }
    // this chunk's weights for output channels n0 .. n0 + nb: per (k, octet)
    // a run of ngb 128-byte core matrices
    {
      const uint4* src = reinterpret_cast<const uint4*>(P.wp) + (size_t)ch * 27 * 2 * ng * 8;
      uint4* dst = reinterpret_cast<uint4*>(sW);
      const int per = ngb * 8;  // uint4 per (k, octet)
      for (int q = tid; q < 27 * 2 * per; q += CT_THREADS) {
        const int ko = q / per, e = q - ko * per;
        dst[q] = src[(size_t)ko * ng * 8 + (n0 / 8) * 8 + e];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
#pragma unroll 1
      for (int k = 0; k < 27; ++k) {
        const int kz = k / 9, ky = (k / 3) % 3, kx = k % 3;
        const uint32_t aoff = (uint32_t)((kz * CT_HX * CT_HY + ky * CT_HX + kx) * 16);
        const uint64_t bd = sdesc(aw + (uint32_t)(k * 2 * ngb * 128), (uint32_t)(ngb * 128), 128);
#pragma unroll
        for (int t3 = 0; t3 < 3; ++t3) {
          const uint64_t ad = sdesc(ax + (uint32_t)(t3 * 2 * CT_PLANE) + aoff, CT_PLANE, CT_HX * 16);
          mma_kf16(tmem, ad, bd, idesc, (ch > 0 || k > 0 || t3 > 0) ? 1u : 0u);
        }
      }
      mma_commit(mb);
    }
    pending = true;
  }
  if (pending && !s_fail && tid == 0) {
    if (mbar_wait(mb, phase))
      pending = false;
    else
      s_fail = 1;
  }
  __syncthreads();
  const bool ok = !s_fail;
  if (!ok) {
    if (tid == 0) {
      if (pending) mbar_wait(mb, phase);  // once more, bounded, before freeing
      atomicOr(P.status, SEA_FLAG_WAIT);
    }
  } else {
    tc_fence_after();
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (row m = lane point),
    // 8-column groups split between warps w < 4 and w >= 4
    const int m = 32 * (warp & 3) + lane;
    const int oy = y0 + (m >> 3), ox = x0 + (m & 7);
    const bool valid = oy < D;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int c8 = warp >> 2; c8 < ngb; c8 += 2) {
      uint32_t r[8];
      tmem_ld8(lane_base + (uint32_t)(c8 * 8), r);
      tmem_wait_ld();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int co = n0 + c8 * 8 + e;
        if (valid && co < P.Cout) {
          float v = __uint_as_float(r[e]) + (P.bias ? P.bias[co] : 0.f);
          if (P.relu) v = fmaxf(v, 0.f);
          P.y[((size_t)b * P.yC + P.yc0 + co) * V + ((size_t)z0 * D + oy) * D + ox] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3x3 layer on the tensor cores:
//
//   dw[co][ci][k] = sum_b sum_p dy[b][co][p] x[b][ci][p + off(k)]
//
// as 27 GEMMs D_k[co][ci] = sum_p A[co][p] B_k[ci][p] whose K dimension is
// the 128 points of a tile.  Both operands are MN-major (8 channels
// contiguous per point): A = the tile's dy, staged point after point
// (rows 16 B apart, one plane per 8 output channels, M = 128 with the
// channels beyond Cout zero); B_k = the haloed input of a 16-channel chunk
// in the forward kernel's layout, shifted by the tap's row offset -- so
// again no im2col copy.  A K step of 16 points is two y-rows of the tile.
// FP32 values enter as two BF16 terms (h + m, 16 significant bits); the
// products h h, h m and m h are accumulated (relative error below 2^-16).
// CTA (g, chunk) of a G x chunks grid takes the tiles g, g + G, ... of the
// whole batch (a fixed assignment) and keeps the 27 accumulators (27 x 16
// columns) in tensor memory over all of them; two staging buffers let the
// next tile be staged while the MMAs of the current one run.  Each CTA
// writes its partial sums; k_conv_dw_reduce adds the G partials in index
// order, so the gradient is deterministic.
// ---------------------------------------------------------------------------
#define DW_THREADS 256
#define DW_APLANE (128 * 16)                            // one 8-channel plane of dy
#define DW_ABYTES (2 * 16 * DW_APLANE)                  // two terms x 16 planes
#define DW_XBYTES (2 * 2 * CT_PLANE)                    // two terms x two octets
#define DW_BUF (DW_ABYTES + DW_XBYTES)

struct ConvDw {
  const float* x;
  int xC, xc0, Cin;
  const float* dy;
  int dyC, dyc0, Cout;
  int D, B, G;
  float* part;  // [chunk][G][27][Cout][16]
  unsigned* status;
};

__device__ __forceinline__ void split2_bf16(float v0, float v1, uint32_t& h, uint32_t& m) {
  const __nv_bfloat162 H = __floats2bfloat162_rn(v0, v1);
  const __nv_bfloat162 Mm = __floats2bfloat162_rn(v0 - __low2float(H), v1 - __high2float(H));
  h = *reinterpret_cast<const uint32_t*>(&H);
  m = *reinterpret_cast<const uint32_t*>(&Mm);
}

__global__ void __launch_bounds__(DW_THREADS, 1) k_conv3_dw_tc(ConvDw P) {
  extern __shared__ unsigned char dw_raw[];
  unsigned char* sb = dw_raw + ((128 - (smem_addr(dw_raw) & 127)) & 127);
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ uint32_t tbase;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = P.D, ntx = D / 8, nty = (D + 15) / 16, ntile = ntx * nty * D;
  const int total = ntile * P.B, g = blockIdx.x, ch = blockIdx.y;
  const size_t V = (size_t)D * D * D;
  const uint32_t mb[2] = {smem_addr(&bars[0]), smem_addr(&bars[1])};
  if (warp == 0) tmem_alloc(&tbase, 512);
  if (tid == 0) {
    mbar_init(mb[0], 1);
    mbar_init(mb[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  // the dy planes of channels beyond Cout stay zero in both buffers
  for (int q = tid; q < 2 * DW_ABYTES / 16; q += DW_THREADS) {
    const int bi = q / (DW_ABYTES / 16), r = q % (DW_ABYTES / 16);
    const int plane = (r * 16 / DW_APLANE) % 16;
    if (8 * plane >= P.Cout)
      *reinterpret_cast<uint4*>(sb + bi * DW_BUF + r * 16) = make_uint4(0, 0, 0, 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  // tcgen05 kind::f16 descriptor: BF16 A and B, both MN-major, M = 128, N = 16
  const uint32_t idesc = idesc_kf16(16, 128, true) | (1u << 15) | (1u << 16);
  const int nplanes = (P.Cout + 7) / 8;
  uint32_t phase[2] = {0, 0};  // thread 0's parities
  int committed[2] = {0, 0};   // commits not yet waited for, per buffer (uniform)
  int i = 0;
  for (int t = g; t < total; t += P.G, ++i) {
    const int buf = i & 1;
    unsigned char* sA = sb + buf * DW_BUF;
    unsigned char* sX = sA + DW_ABYTES;
    if (committed[buf]) {  // the MMAs of two tiles ago read this buffer
      if (tid == 0) {
        if (mbar_wait(mb[buf], phase[buf]))
          phase[buf] ^= 1;
        else
          s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      committed[buf] = 0;
    }
    const int b = t / ntile;
    int r = t % ntile;
    const int x0 = (r % ntx) * 8;
    r /= ntx;
    const int y0 = (r % nty) * 16, z0 = r / nty;
    // dy of the tile: item = (plane, point m), 8 channels
    for (int it = tid; it < nplanes * 128; it += DW_THREADS) {
      const int pl = it / 128, m = it % 128;
      const int oy = y0 + (m >> 3), ox = x0 + (m & 7);
      const bool in = oy < D;
      const size_t pofs = ((size_t)z0 * D + (in ? oy : 0)) * D + ox;
      uint32_t w[2][4];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const int co = 8 * pl + 2 * c2;
        const float v0 = (in && co < P.Cout) ? P.dy[((size_t)b * P.dyC + P.dyc0 + co) * V + pofs] : 0.f;
        const float v1 =
            (in && co + 1 < P.Cout) ? P.dy[((size_t)b * P.dyC + P.dyc0 + co + 1) * V + pofs] : 0.f;
        split2_bf16(v0, v1, w[0][c2], w[1][c2]);
      }
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2)
        *reinterpret_cast<uint4*>(sA + (t2 * 16 + pl) * DW_APLANE + m * 16) =
            make_uint4(w[t2][0], w[t2][1], w[t2][2], w[t2][3]);
    }
    // the haloed input of channels 16 ch .. + 15
    for (int it = tid; it < 2 * CT_ROWS; it += DW_THREADS) {
      const int o = it / CT_ROWS, row = it - o * CT_ROWS;
      const int hx = row % CT_HX, hy = (row / CT_HX) % CT_HY, hz = row / (CT_HX * CT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool in = gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D;
      const size_t pofs = in ? ((size_t)gz * D + gy) * D + gx : 0;
      uint32_t w[2][4];
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) {
        const int ci = 16 * ch + 8 * o + 2 * c2;
        const float v0 = (in && ci < P.Cin) ? P.x[((size_t)b * P.xC + P.xc0 + ci) * V + pofs] : 0.f;
        const float v1 =
            (in && ci + 1 < P.Cin) ? P.x[((size_t)b * P.xC + P.xc0 + ci + 1) * V + pofs] : 0.f;
        split2_bf16(v0, v1, w[0][c2], w[1][c2]);
      }
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2)
        *reinterpret_cast<uint4*>(sX + (t2 * 2 + o) * CT_PLANE + row * 16) =
            make_uint4(w[t2][0], w[t2][1], w[t2][2], w[t2][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t aa = smem_addr(sA), ax = smem_addr(sX);
#pragma unroll 1
      for (int k = 0; k < 27; ++k) {
        const int kz = k / 9, ky = (k / 3) % 3, kx = k % 3;
        const uint32_t aoff = (uint32_t)((kz * CT_HX * CT_HY + ky * CT_HX + kx) * 16);
#pragma unroll 1
        for (int st = 0; st < 8; ++st) {  // K step: points 16 st .. 16 st + 15 (y rows 2 st, 2 st + 1)
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {  // term pairs h h, h m, m h
            const int ta = pr == 2 ? 1 : 0, tb = pr == 1 ? 1 : 0;
            // MN-major operands: lbo = byte distance of K-adjacent core
            // matrices (the next 8 points), sbo = of M/N-adjacent ones (the
            // next 8 channels)
            const uint64_t ad = sdesc(aa + (uint32_t)(ta * 16 * DW_APLANE + st * 256), 128, DW_APLANE);
            const uint64_t bd =
                sdesc(ax + (uint32_t)(tb * 2 * CT_PLANE) + aoff + (uint32_t)(st * 2 * CT_HX * 16),
                      CT_HX * 16, CT_PLANE);
            mma_kf16(tmem + (uint32_t)(k * 16), ad, bd, idesc, (i > 0 || st > 0 || pr > 0) ? 1u : 0u);
          }
        }
      }
      mma_commit(mb[buf]);
    }
    committed[buf] = 1;
  }
  // the last tiles' MMAs
  for (int q = 0; q < 2; ++q) {
    const int bq = (i + q) & 1;  // oldest first
    if (committed[bq] && !s_fail) {
      if (tid == 0) {
        if (mbar_wait(mb[bq], phase[bq])) {
          phase[bq] ^= 1;
        } else {
          s_fail = 1;
        }
      }
      __syncthreads();
      if (!s_fail) committed[bq] = 0;
    }
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      for (int q = 0; q < 2; ++q)
        if (committed[q]) mbar_wait(mb[q], phase[q]);  // once more, bounded
      atomicOr(P.status, SEA_FLAG_WAIT);
    }
  } else if (warp < 4) {
    tc_fence_after();
    const int co = 32 * warp + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    float* dst = P.part + (((size_t)ch * P.G + g) * 27) * P.Cout * 16;
    for (int k = 0; k < 27; ++k) {
      uint32_t v[16];
      tmem_ld8(lane_base + (uint32_t)(k * 16), v);
      tmem_ld8(lane_base + (uint32_t)(k * 16 + 8), v + 8);
      tmem_wait_ld();
      if (co < P.Cout)
#pragma unroll
        for (int c = 0; c < 16; ++c)
          dst[((size_t)k * P.Cout + co) * 16 + c] = i > 0 ? __uint_as_float(v[c]) : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// dw[co][ci][k] = sum over g (in index order) of the CTAs' partial sums.
__global__ void k_conv_dw_reduce(const float* __restrict__ part, int Cout, int Cin, int G,
                                 float* __restrict__ dw) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Cout * Cin * 27) return;
  const int k = q % 27, ci = (q / 27) % Cin, co = q / (27 * Cin);
  const int ch = ci / 16, c = ci % 16;
  const float* p = part + ((size_t)ch * G * 27 + k) * Cout * 16 + (size_t)co * 16 + c;
  const size_t stride = (size_t)27 * Cout * 16;
  float s = 0.f;
  for (int gg = 0; gg < G; ++gg) s += p[gg * stride];
  dw[q] = s;
}

// db[co] = sum_b sum_p dy[b][dyc0 + co][p]: CTA per co, fixed-order reduction.
__global__ void __launch_bounds__(256)
    k_bias_grad(const float* __restrict__ dy, int dyC, int dyc0, size_t V, int B,
                float* __restrict__ db) {
  const int co = blockIdx.x;
  float s = 0.f;
  for (size_t e = threadIdx.x; e < (size_t)B * V; e += blockDim.x) {
    const int b = (int)(e / V);
    s += dy[((size_t)b * dyC + dyc0 + co) * V + e % V];
  }
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[co] = red[0];
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
  // tensor-core layouts of a 3x3x3 layer's BF16 weights (k_conv_wprep):
  // forward (N = cout padded to 16) and transposed for the data gradient
  // (N = cin padded to 16); offsets in sea_unet::wp
  int npad_f = 0, npad_t = 0;
  long long wpf_off = 0, wpt_off = 0;
};

struct sea_unet {
  int width = 16, device = 0, bmax = 32;
  cudaStream_t stream = nullptr;
  std::vector<UnLayer> L;
  long long nparam = 0;
  float *master = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  __nv_bfloat16 *wb = nullptr, *wp = nullptr;  // BF16 weights; their tensor-core layouts
  long long nwp = 0;
  float* dwpart = nullptr;      // the weight-gradient kernel's per-CTA partial sums
  int nsm = 0;
  unsigned* status = nullptr;   // device status word of the model's own calls
  unsigned* st_use = nullptr;   // the word the kernels report to (the model's or a context's)
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

// Synchronize the model's stream and check its status word (a bounded
// tensor-core wait that expired): the word is cleared for the next call.
sea_status un_sync(sea_unet* u) {
  unsigned st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, u->status, sizeof(unsigned), cudaMemcpyDeviceToHost, u->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) return un_fail(u, SEA_ERR_CUDA, cudaGetErrorString(e));
  if (st & SEA_FLAG_WAIT) {
    cudaMemsetAsync(u->status, 0, sizeof(unsigned), u->stream);
    return un_fail(u, SEA_ERR_CUDA, "a tensor-core completion wait timed out");
  }
  return SEA_OK;
}

int pad16(int n) { return (n + 15) / 16 * 16; }

size_t conv_smem(int npad) {
  return 128 + CT_XBYTES + (size_t)27 * 2 * (std::min(npad, CT_NBLK) / 8) * 128;
}

// Tensor-core layouts of every 3x3x3 layer's BF16 weights (after any change
// of u->wb).
void prep_weights(sea_unet* u) {
  for (const UnLayer& a : u->L) {
    if (a.k != 3) continue;
    const long long nf = (long long)pad16(a.cin) * a.npad_f * 27;
    sea::k_conv_wprep<<<grid1(nf), 256, 0, u->stream>>>(u->wb + a.w_off, a.cout, a.cin, 0, a.npad_f,
                                                        u->wp + a.wpf_off);
    const long long nt = (long long)pad16(a.cout) * a.npad_t * 27;
    sea::k_conv_wprep<<<grid1(nt), 256, 0, u->stream>>>(u->wb + a.w_off, a.cout, a.cin, 1, a.npad_t,
                                                        u->wp + a.wpt_off);
  }
}

// y (slice yc0 of yC channels) = act(conv3 of x's slice) for layer l, or for
// transpose = true the data gradient: the transposed convolution of the
// layer (cin and cout exchanged, flipped taps), no bias, no activation.
void conv3_tc(sea_unet* u, int l, bool transpose, const float* x, int xC, int xc0, float* y,
              int yC, int yc0, int D, int B, int relu) {
  const UnLayer& a = u->L[l];
  sea::ConvTc P;
  P.x = x;
  P.xC = xC;
  P.xc0 = xc0;
  P.Cin = transpose ? a.cout : a.cin;
  P.wp = u->wp + (transpose ? a.wpt_off : a.wpf_off);
  P.npad = transpose ? a.npad_t : a.npad_f;
  P.bias = transpose ? nullptr : u->master + a.b_off;
  P.y = y;
  P.yC = yC;
  P.yc0 = yc0;
  P.Cout = transpose ? a.cin : a.cout;
  P.D = D;
  P.relu = relu;
  P.status = u->st_use;
  const int tiles = (D / 8) * ((D + 15) / 16) * D;
  const int nzb = (P.npad + CT_NBLK - 1) / CT_NBLK;
  sea::k_conv3_tc<<<dim3(tiles, B, nzb), CT_THREADS, conv_smem(P.npad), u->stream>>>(P);
}

void conv3(sea_unet* u, const float* x, int xC, int xc0, int l, float* y, int yC, int yc0, int D,
           int B, int relu) {
  conv3_tc(u, l, false, x, xC, xc0, y, yC, yc0, D, B, relu);
}

// dx (slice of a tensor with xC channels) = transposed convolution of dy
void conv3_dx(sea_unet* u, int l, const float* dy, int dyC, float* dx, int xC, int xc0, int D,
              int B) {
  conv3_tc(u, l, true, dy, dyC, 0, dx, xC, xc0, D, B, 0);
}

// Grid of the weight-gradient kernel: G CTAs per 16-channel chunk, about one
// CTA per SM in all (each holds the SM's 512 tensor-memory columns).
int dw_grid(const sea_unet* u, int cin, int D, int B) {
  const int nch = (cin + 15) / 16;
  const int tiles = (D / 8) * ((D + 15) / 16) * D * B;
  return std::max(1, std::min(tiles, (u->nsm + nch - 1) / nch));
}

size_t dw_part_floats(const sea_unet* u, const UnLayer& a, int D, int B) {
  return (size_t)((a.cin + 15) / 16) * dw_grid(u, a.cin, D, B) * 27 * a.cout * 16;
}

// u->grad of layer l's weights and bias from the layer input x (slice xc0 of
// xC channels) and the output gradient dy (slice dyc0 of dyC channels).
void conv3_dw(sea_unet* u, int l, const float* x, int xC, int xc0, const float* dy, int dyC,
              int dyc0, int D, int B) {
  const UnLayer& a = u->L[l];
  sea::ConvDw P;
  P.x = x;
  P.xC = xC;
  P.xc0 = xc0;
  P.Cin = a.cin;
  P.dy = dy;
  P.dyC = dyC;
  P.dyc0 = dyc0;
  P.Cout = a.cout;
  P.D = D;
  P.B = B;
  P.G = dw_grid(u, a.cin, D, B);
  P.part = u->dwpart;
  P.status = u->st_use;
  const int nch = (a.cin + 15) / 16;
  sea::k_conv3_dw_tc<<<dim3(P.G, nch), DW_THREADS, 128 + 2 * DW_BUF, u->stream>>>(P);
  sea::k_conv_dw_reduce<<<grid1((size_t)a.cout * a.cin * 27), 256, 0, u->stream>>>(
      u->dwpart, a.cout, a.cin, P.G, u->grad + a.w_off);
  sea::k_bias_grad<<<a.cout, 256, 0, u->stream>>>(dy, dyC, dyc0, (size_t)D * D * D, B,
                                                   u->grad + a.b_off);
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
  conv3_dw(u, 9, u->d1a, c, 0, u->g32a, c, 0, 32, B);
  conv3_dx(u, 9, u->g32a, c, u->g32b, c, 0, 32, B);
  // d1a = relu(conv8(cat1))
  relu_bwd(u, u->g32b, c, 0, u->d1a, c, 0, c, 32, B);
  conv3_dw(u, 8, u->cat1, 3 * c, 0, u->g32b, c, 0, 32, B);
  conv3_dx(u, 8, u->g32b, c, u->gcat1, 3 * c, 0, 32, B);
  // cat1[0..2c) = up(d2b)
  sea::k_up_bwd<<<grid1((size_t)B * 2 * c * V16), 256, 0, u->stream>>>(u->gcat1, 3 * c, 0, u->g16a,
                                                                       2 * c, 16, B);
  // d2b = relu(conv7(d2a))
  relu_bwd(u, u->g16a, 2 * c, 0, u->d2b, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 7, u->d2a, 2 * c, 0, u->g16a, 2 * c, 0, 16, B);
  conv3_dx(u, 7, u->g16a, 2 * c, u->g16b, 2 * c, 0, 16, B);
  // d2a = relu(conv6(cat2))
  relu_bwd(u, u->g16b, 2 * c, 0, u->d2a, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 6, u->cat2, 6 * c, 0, u->g16b, 2 * c, 0, 16, B);
  conv3_dx(u, 6, u->g16b, 2 * c, u->gcat2, 6 * c, 0, 16, B);
  // cat2[0..4c) = up(b5)
  sea::k_up_bwd<<<grid1((size_t)B * 4 * c * V8), 256, 0, u->stream>>>(u->gcat2, 6 * c, 0, u->g8a,
                                                                      4 * c, 8, B);
  // b5 = relu(conv5(b4)), b4 = relu(conv4(p2))
  relu_bwd(u, u->g8a, 4 * c, 0, u->b5, 4 * c, 0, 4 * c, 8, B);
  conv3_dw(u, 5, u->b4, 4 * c, 0, u->g8a, 4 * c, 0, 8, B);
  conv3_dx(u, 5, u->g8a, 4 * c, u->g8b, 4 * c, 0, 8, B);
  relu_bwd(u, u->g8b, 4 * c, 0, u->b4, 4 * c, 0, 4 * c, 8, B);
  conv3_dw(u, 4, u->p2, 2 * c, 0, u->g8b, 4 * c, 0, 8, B);
  conv3_dx(u, 4, u->g8b, 4 * c, u->g8a, 2 * c, 0, 8, B);  // d p2
  // p2 = pool(cat2[4c..6c)): add into the skip-2 gradient slice of gcat2
  sea::k_pool_bwd<<<grid1((size_t)B * 2 * c * V16), 256, 0, u->stream>>>(u->g8a, u->gcat2, 6 * c,
                                                                        4 * c, 2 * c, 16, B, 1);
  // skip 2 = relu(conv3(e2a))
  relu_bwd(u, u->gcat2, 6 * c, 4 * c, u->cat2, 6 * c, 4 * c, 2 * c, 16, B);
  conv3_dw(u, 3, u->e2a, 2 * c, 0, u->gcat2, 6 * c, 4 * c, 16, B);
  conv3_tc(u, 3, true, u->gcat2, 6 * c, 4 * c, u->g16a, 2 * c, 0, 16, B, 0);
  // e2a = relu(conv2(p1))
  relu_bwd(u, u->g16a, 2 * c, 0, u->e2a, 2 * c, 0, 2 * c, 16, B);
  conv3_dw(u, 2, u->p1, c, 0, u->g16a, 2 * c, 0, 16, B);
  conv3_dx(u, 2, u->g16a, 2 * c, u->g16b, c, 0, 16, B);  // d p1
  // p1 = pool(cat1[2c..3c)): add into the skip-1 gradient slice of gcat1
  sea::k_pool_bwd<<<grid1((size_t)B * c * V32), 256, 0, u->stream>>>(u->g16b, u->gcat1, 3 * c, 2 * c,
                                                                     c, 32, B, 1);
  // skip 1 = relu(conv1(e1a))
  relu_bwd(u, u->gcat1, 3 * c, 2 * c, u->cat1, 3 * c, 2 * c, c, 32, B);
  conv3_dw(u, 1, u->e1a, c, 0, u->gcat1, 3 * c, 2 * c, 32, B);
  conv3_tc(u, 1, true, u->gcat1, 3 * c, 2 * c, u->g32a, c, 0, 32, B, 0);
  // e1a = relu(conv0(in))
  relu_bwd(u, u->g32a, c, 0, u->e1a, c, 0, c, 32, B);
  conv3_dw(u, 0, in, 2, 0, u->g32a, c, 0, 32, B);
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
  if (u->wp) cudaFree(u->wp);
  if (u->dwpart) cudaFree(u->dwpart);
  if (u->status) cudaFree(u->status);
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
  long long off = 0;
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
    if (l.k == 3) {
      l.npad_f = pad16(l.cout);
      l.npad_t = pad16(l.cin);
      l.wpf_off = u->nwp;
      u->nwp += (long long)pad16(l.cin) * l.npad_f * 27;
      l.wpt_off = u->nwp;
      u->nwp += (long long)pad16(l.cout) * l.npad_t * 27;
    }
    u->L.push_back(l);
  }
  u->nparam = off;
  cudaDeviceGetAttribute(&u->nsm, cudaDevAttrMultiProcessorCount, u->device);
  if (u->nsm < 1) u->nsm = 1;
  size_t dw_max = 1;
  {
    const int Ds[10] = {32, 32, 16, 16, 8, 8, 16, 16, 32, 32};
    for (int l = 0; l < 10; ++l) dw_max = std::max(dw_max, dw_part_floats(u, u->L[l], Ds[l], u->bmax));
  }
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
            alloc((void**)&u->wb, off * 2) && alloc((void**)&u->wp, u->nwp * 2) &&
            alloc((void**)&u->status, 16) && alloc((void**)&u->dwpart, dw_max * 4) &&
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
  prep_weights(u);
  u->st_use = u->status;
  if (cudaMemsetAsync(u->status, 0, 16, u->stream) != cudaSuccess ||
      cudaFuncSetAttribute(sea::k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)conv_smem(CT_NBLK)) != cudaSuccess ||
      cudaFuncSetAttribute(sea::k_conv3_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           128 + 2 * DW_BUF) != cudaSuccess ||
      cudaStreamSynchronize(u->stream) != cudaSuccess) {
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
      prep_weights(u);
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
  return un_sync(u);
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
  const sea_status st = un_sync(u);
  if (st != SEA_OK) return st;
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
    prep_weights(u);
  }
  if (steps > 0) cudaMemcpyAsync(&l, u->dloss, 8, cudaMemcpyDeviceToHost, u->stream);
  const sea_status st = un_sync(u);
  if (st != SEA_OK) return st;
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
  // The model runs on the context's stream here and reports to its status word.
  cudaStream_t saved = u->stream;
  u->stream = c->stream;
  u->st_use = (unsigned*)c->status.p;
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
  u->st_use = u->status;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // smooth the guesses' high-frequency error before the CG
  return launch_smooth(c, 4, 2.0 / 3.0);
}

}  // namespace sea
