// ace.cu -- adaptively compressed exchange (Sec. II C, Eq. Vace; App. A).
//
// W = V_xx Phi is exactly zero outside the accumulation windows of each
// orbital (Eq. tDxx), so every contraction with W runs over the grid tiles
// (8 x 4 x 4 points) that those windows touch; the result is the dense
// definition's, only without the exact zeros:
//   M_ij = <phi_i|W_j> = dV sum over tiles of W_j of phi_i W_j
//   Mbar = (M + M^T)/2, -Mbar = L L^T (Cholesky, one CTA), L^-1
//   Xi = W L^-T                              (materialized on request)
//   V^ACE psi = -Xi Xi^T psi dV = -W L^-T L^-1 (W^T psi dV)
// The contractions are FP64 FMA on the CUDA cores: on this part the measured
// FP64 FMA rate is above the FP64 tensor (DMMA) rate.
#include "sea_internal.cuh"

namespace sea {


__device__ __forceinline__ bool cyc_meets(int s, int L, int a, int b, int n) {
  // cyclic [s, s+L) (s wrapped) meets [a, b) (0 <= a < b <= n)
  if (L >= n) return true;
  return (wrapi(s - a, n) < b - a) || (wrapi(a - s, n) < L);
}

// Covered range [lo, hi) of the tile interval [a, b) by the cyclic window
// [s, s+L) on a ring of n points (lo >= hi: none).
// The window is [s, s + L) and, if it passes n, [0, s + L - n) (s in
// [0, n), L < n); the covered range spans the parts meeting [a, b).
__device__ __forceinline__ void cyc_cover(int s, int L, int a, int b, int n, int* lo, int* hi) {
  if (L >= n) {
    *lo = a;
    *hi = b;
    return;
  }
  int l = b, h = a;
  const int l1 = max(a, s), h1 = min(b, s + L);
  if (l1 < h1) {
    l = l1;
    h = h1;
  }
  const int h2 = min(b, s + L - n);  // the wrapped part starts at 0 <= a
  if (a < h2) {
    l = a;
    h = max(h, h2);
  }
  *lo = l;
  *hi = h;
}

// inc[o][T] = 1 if any entry window of orbital o touches tile T, and
// sub[o][T] = the bounding box, in tile coordinates, of the union of those
// windows inside the tile, packed x0 | x1 << 4 | y0 << 8 | y1 << 12 |
// z0 << 16 | z1 << 20 (W_o is exactly zero in the tile outside it).
__global__ void k_tile_incidence(const Entry* __restrict__ ent, const int* __restrict__ eptr,
                                 int n_orb, TileGeom G, int n_tiles, int dense,
                                 int* __restrict__ inc, int* __restrict__ sub) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_orb * n_tiles) return;
  const int o = (int)(t / n_tiles), T = (int)(t % n_tiles);
  const int txi = T % G.ntx, tyi = (T / G.ntx) % G.nty, tzi = T / (G.ntx * G.nty);
  const int ax = txi * TX, bx = min(G.nx, ax + TX);
  const int ay = tyi * TY, by = min(G.ny, ay + TY);
  const int az = tzi * TZ, bz = min(G.nz, az + TZ);
  if (dense) {  // W given by the caller: no known support, the whole tile
    inc[t] = 1;
    sub[t] = 0 | ((bx - ax) << 4) | (0 << 8) | ((by - ay) << 12) | (0 << 16) | ((bz - az) << 20);
    return;
  }
  int x0 = TX, x1 = 0, y0 = TY, y1 = 0, z0 = TZ, z1 = 0;
  for (int k = eptr[o]; k < eptr[o + 1]; ++k) {
    const Entry e = ent[k];
    int lx, hx, ly, hy, lz, hz;
    cyc_cover(wrapi(e.ws[0], G.nx), e.wl[0], ax, bx, G.nx, &lx, &hx);
    if (lx >= hx) continue;
    cyc_cover(wrapi(e.ws[1], G.ny), e.wl[1], ay, by, G.ny, &ly, &hy);
    if (ly >= hy) continue;
    cyc_cover(wrapi(e.ws[2], G.nz), e.wl[2], az, bz, G.nz, &lz, &hz);
    if (lz >= hz) continue;
    x0 = min(x0, lx - ax);
    x1 = max(x1, hx - ax);
    y0 = min(y0, ly - ay);
    y1 = max(y1, hy - ay);
    z0 = min(z0, lz - az);
    z1 = max(z1, hz - az);
  }
  const int hit = x1 > x0;
  inc[t] = hit;
  sub[t] = hit ? (x0 | (x1 << 4) | (y0 << 8) | (y1 << 12) | (z0 << 16) | (z1 << 20)) : 0;
}

// Tile-major lists: one warp per tile, orbitals ascending (ballot
// compaction keeps the order).  mode 0 counts, mode 1 writes the list and
// the incidence index gidx[o][T].
__global__ void k_tile_lists(const int* __restrict__ inc, const int* __restrict__ sub, int n_orb,
                             int n_tiles, int mode, int* __restrict__ cnt,
                             const int* __restrict__ ptr, int* __restrict__ list,
                             int* __restrict__ lsub, int* __restrict__ gidx) {
  const int T = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (T >= n_tiles) return;  // warp-uniform
  int c = 0;
  const int base = mode ? ptr[T] : 0;
  for (int o0 = 0; o0 < n_orb; o0 += 32) {
    const int o = o0 + lane;
    const size_t q = (size_t)o * n_tiles + T;
    const bool hit = o < n_orb && inc[q];
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (mode && o < n_orb) {
      if (hit) {
        const int pos = base + c + __popc(bal & ((1u << lane) - 1u));
        list[pos] = o;
        lsub[pos] = sub[q];
        gidx[q] = pos;
      } else {
        gidx[q] = -1;
      }
    }
    c += __popc(bal);
  }
  if (!mode && lane == 0) cnt[T] = c;
}

// Orbital-major lists: one warp per orbital, tiles ascending (ballot
// compaction keeps the order), with the incidence index of each
// (orbital, tile).  mode 0 counts, mode 1 writes.
__global__ void k_orb_lists(const int* __restrict__ gidx, int n_orb, int n_tiles, int mode,
                            int* __restrict__ cnt, const int* __restrict__ ptr,
                            int* __restrict__ list, int* __restrict__ slot) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n_orb) return;
  int c = 0;
  const int base = mode ? ptr[o] : 0;
  for (int T0 = 0; T0 < n_tiles; T0 += 128) {  // four chunks of 32 tiles per step
    int g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int T = T0 + 32 * u + lane;
      g[u] = T < n_tiles ? gidx[(size_t)o * n_tiles + T] : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned bal = __ballot_sync(0xffffffffu, g[u] >= 0);
      if (mode && g[u] >= 0) {
        const int pos = base + c + __popc(bal & ((1u << lane) - 1u));
        list[pos] = T0 + 32 * u + lane;
        slot[pos] = g[u];
      }
      c += __popc(bal);
    }
  }
  if (!mode && lane == 0) cnt[o] = c;
}

__global__ void k_scan_small(const int* __restrict__ in, int n, int* __restrict__ out,
                             int* __restrict__ tot) {
  __shared__ long long part[32];
  const int T = blockDim.x, chunk = (n + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(n, b + chunk);
  long long s = 0;
  for (int x = b; x < e; ++x) s += in[x];
  long long acc = 0;
  long long pos = block_exscan_ll(s, part, &acc);
  if (threadIdx.x == 0) *tot = (int)acc;
  for (int x = b; x < e; ++x) {
    out[x] = (int)pos;
    pos += in[x];
  }
  if (threadIdx.x == T - 1) out[n] = (int)pos;
}

__global__ void k_max_int(const int* __restrict__ in, int n, int* __restrict__ out) {
  __shared__ int part[1024];
  int m = 0;
  for (int x = threadIdx.x; x < n; x += blockDim.x) m = max(m, in[x]);
  part[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)blockDim.x; ++t) m = max(m, part[t]);
    *out = max(part[0], m);
  }
}


// partial[(tptr[T] + s) * m + a] = sum_{r in T} A[a][r] W[list[s]][r].
// CTA per (tile, chunk of 64 rows of A).  The tile's 128 points of the 64
// A rows and of up to 32 W rows sit in shared memory; a work unit is
// (W row, half of the A rows), units are dealt to warps in a warp-uniform
// loop (no predicated FMAs: on this part a predicated-off FP64 FMA still
// costs FP64 pipe time), each lane one A row; the dot product runs over the
// W row's sub-box of the tile only (W is exactly zero outside it), with
// four independent FMA chains along x.
#define GA 64
#define GJB 32
#define GROW (TP + 1)
#define GRAM_SMEM ((size_t)(GA + GJB) * GROW * sizeof(double))
__global__ void __launch_bounds__(256, 2)
    k_gram_partial(const double* __restrict__ A, int m, const double* __restrict__ W,
                   TileGeom G, size_t ng, const int* __restrict__ tptr,
                   const int* __restrict__ tlist, const int* __restrict__ tsub,
                   double* __restrict__ partial) {
  const int T = blockIdx.x;
  const int a0 = blockIdx.y * GA;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (nJ == 0) return;
  extern __shared__ double gsm[];
  double* As = gsm;               // [GA][GROW]
  double* Ws = gsm + GA * GROW;   // [GJB][GROW]
  __shared__ long long addr[TP];
  __shared__ int wrow[GJB];
  for (int r = threadIdx.x; r < TP; r += blockDim.x) addr[r] = tile_point(G, T, r);
  __syncthreads();
  for (int idx = threadIdx.x; idx < GA * TP; idx += blockDim.x) {
    const int a = idx / TP, pt = idx % TP;
    const long long g = addr[pt];
    As[a * GROW + pt] = (a0 + a < m && g >= 0) ? A[(size_t)(a0 + a) * ng + g] : 0.0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int jb = 0; jb < nJ; jb += GJB) {
    const int nj = min(GJB, nJ - jb);
    __syncthreads();
    if (threadIdx.x < nj) wrow[threadIdx.x] = tlist[j0 + jb + threadIdx.x];
    __syncthreads();
    for (int idx = threadIdx.x; idx < nj * TP; idx += blockDim.x) {
      const int jl = idx / TP, pt = idx % TP;
      const long long g = addr[pt];
      Ws[jl * GROW + pt] = g >= 0 ? W[(size_t)wrow[jl] * ng + g] : 0.0;
    }
    __syncthreads();
    for (int u = warp; u < 2 * nj; u += nwarp) {
      const int jl = u >> 1, ah = u & 1;
      const double* ar = As + (ah * 32 + lane) * GROW;
      const double* wr = Ws + jl * GROW;
      const int sb = tsub[j0 + jb + jl];
      const int x0 = sb & 15, x1 = (sb >> 4) & 15, y0 = (sb >> 8) & 15, y1 = (sb >> 12) & 15,
                z0 = (sb >> 16) & 15, z1 = (sb >> 20) & 15;
      double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
      for (int z = z0; z < z1; ++z)
        for (int y = y0; y < y1; ++y) {
          const int base = (z * TY + y) * TX;
          int x = x0;
          for (; x + 4 <= x1; x += 4) {
            c0 = fma(ar[base + x], wr[base + x], c0);
            c1 = fma(ar[base + x + 1], wr[base + x + 1], c1);
            c2 = fma(ar[base + x + 2], wr[base + x + 2], c2);
            c3 = fma(ar[base + x + 3], wr[base + x + 3], c3);
          }
          for (; x < x1; ++x) c0 = fma(ar[base + x], wr[base + x], c0);
        }
      const int a = a0 + ah * 32 + lane;
      if (a < m) partial[(size_t)(j0 + jb + jl) * m + a] = (c0 + c1) + (c2 + c3);
    }
  }
}

// ---------------------------------------------------------------------------
// Mixed form of the expansion W H (k_tile_expand_x): FP64 operands split into
// FP32 pairs (v = hi + lo, hi = fl32(v), lo = fl32(v - hi)), each product
// formed as hi*hi exactly (FMA residual) plus the two cross terms, and
// summed with an error-free addition into a (sum, compensation) pair of
// FP32 values: about 44 significant bits, at the FP32 issue rate, which on
// this part is 64x the FP64 rate.  (The mixed form's contraction with W,
// M = Phi^T W and W^T psi, runs on the tensor cores: gram_tc.cu.)
// ---------------------------------------------------------------------------
struct CompF {
  float s, c;
  __device__ CompF() : s(0.f), c(0.f) {}
  // add (ah + al)(bh + bl), dropping al*bl
  __device__ __forceinline__ void add_prod(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    const float x = fmaf(ah, bl, al * bh);
    const float t = s + p;
    const float z = t - s;
    const float err = (s - (t - z)) + (p - z);
    s = t;
    c += (err + e) + x;
  }
  // sgn * (s + c) as FP64, with integer operations only: both terms as
  // fixed-point integers on the larger one's exponent (truncating the
  // smaller one's bits below 2^-38 of it), then one rounding to nearest.
  // FP32 subnormals count as zero.
  __device__ __forceinline__ double value(bool negate) const {
    const unsigned bs = __float_as_uint(s), bc = __float_as_uint(c);
    const int es = (int)((bs >> 23) & 0xFF), ec = (int)((bc >> 23) & 0xFF);
    const int E = max(es, ec);
    if (E == 0) return 0.0;
    auto fixed = [&](unsigned b, int e) -> long long {
      if (e == 0) return 0;
      const int sh = E - e;
      if (sh > 62) return 0;
      const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u) << 38;
      const long long v = m >> sh;
      return (b >> 31) ? -v : v;
    };
    long long X = fixed(bs, es) + fixed(bc, ec);
    if (negate) X = -X;
    return scaled_i64(X, E - 150 - 38);
  }
};


// Mixed form of k_tile_expand (same splitting and compensated sums).
__global__ void __launch_bounds__(256)
    k_tile_expand_x(const double* __restrict__ W, TileGeom G, size_t ng,
                    const int* __restrict__ tptr, const int* __restrict__ tlist,
                    const int* __restrict__ tsub, const double* __restrict__ H, long long hj,
                    long long hv, int m, double sign, int skip_upto, double* __restrict__ out) {
  const int T = blockIdx.x;
  const int v0 = blockIdx.y * 32;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (nJ <= skip_upto) return;  // done by the tensor-core expansion
  extern __shared__ float2 Hx[];  // [nJ][32]
  for (int idx = threadIdx.x; idx < nJ * 32; idx += blockDim.x) {
    const int jl = idx / 32, vl = idx % 32;
    Hx[idx] = split64((v0 + vl < m) ? H[(long long)tlist[j0 + jl] * hj + (long long)(v0 + vl) * hv]
                                    : 0.0);
  }
  __syncthreads();
  const int pt = threadIdx.x % TP, vh = threadIdx.x / TP;
  const long long g = tile_point(G, T, pt);
  CompF acc[16];
  const int pz = pt / (TX * TY), py = (pt / TX) % TY, px = pt % TX;  // pz: one per warp
  // W value of list entry jl at this point (0 outside its sub-box); the
  // next entry's value is loaded while the current one is used
  auto fetch = [&](int jl) {
    const int sb = tsub[j0 + jl];
    const bool in = px >= (sb & 15) && px < ((sb >> 4) & 15) && py >= ((sb >> 8) & 15) &&
                    py < ((sb >> 12) & 15) && pz >= ((sb >> 16) & 15) && pz < ((sb >> 20) & 15);
    return (g >= 0 && in) ? W[(size_t)tlist[j0 + jl] * ng + g] : 0.0;
  };
  double wnext = nJ > 0 ? fetch(0) : 0.0;
  for (int jl = 0; jl < nJ; ++jl) {
    const double wv = wnext;
    if (jl + 1 < nJ) wnext = fetch(jl + 1);
    const int sb = tsub[j0 + jl];
    if (pz < ((sb >> 16) & 15) || pz >= ((sb >> 20) & 15)) continue;  // warp-uniform
    const float2 w = split64(wv);
    const float2* hrow = Hx + jl * 32 + vh * 16;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const float2 hh = hrow[u];
      acc[u].add_prod(w.x, w.y, hh.x, hh.y);
    }
  }
  if (g < 0) return;
  const bool negate = sign < 0.0;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int v = v0 + vh * 16 + u;
    if (v < m) out[(size_t)v * ng + g] = acc[u].value(negate);
  }
}

// out[a * sa + o * so] = scale * sum over the tiles of o of partial[slot][a].
// A CTA per (orbital o, 64 values of a): its four thread groups z take the
// slots z, z + 4, z + 8, ... of o's list (eight loads in flight each, added
// in list order), and the four sums are added in the order z = 0, 1, 2, 3.
constexpr int GR_A = 64, GR_Z = 4;
__global__ void __launch_bounds__(GR_A * GR_Z)
    k_gram_reduce(const double* __restrict__ partial, int m, int n_orb,
                  const int* __restrict__ optr, const int* __restrict__ oslot, double scale,
                  double* __restrict__ out, int sa, int so) {
  __shared__ double red[GR_Z][GR_A];
  const int o = blockIdx.y, x = threadIdx.x % GR_A, z = threadIdx.x / GR_A;
  const int a = blockIdx.x * GR_A + x;
  double s = 0.0;
  if (a < m) {
    int k = optr[o] + z;
    const int k1 = optr[o + 1];
    for (; k + 7 * GR_Z < k1; k += 8 * GR_Z) {
      double p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] = partial[(size_t)oslot[k + u * GR_Z] * m + a];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += p[u];
    }
    for (; k < k1; k += GR_Z) s += partial[(size_t)oslot[k] * m + a];
  }
  red[z][x] = s;
  __syncthreads();
  if (z == 0 && a < m)
    out[(size_t)a * sa + (size_t)o * so] = scale * (((red[0][x] + red[1][x]) + red[2][x]) + red[3][x]);
}

// The same sums in double-float for the mixed form (the partials split
// exactly to FP32 pairs, sums on the FP32 pipes; the FP64 adds of the form
// above bound it there), one rounding to FP64 before the scaling.
__global__ void __launch_bounds__(GR_A * GR_Z)
    k_gram_reduce_df(const double* __restrict__ partial, int m, int n_orb,
                     const int* __restrict__ optr, const int* __restrict__ oslot, double scale,
                     double* __restrict__ out, int sa, int so) {
  __shared__ DF red[GR_Z][GR_A];
  const int o = blockIdx.y, x = threadIdx.x % GR_A, z = threadIdx.x / GR_A;
  const int a = blockIdx.x * GR_A + x;
  DF s{0.f, 0.f};
  if (a < m) {
    int k = optr[o] + z;
    const int k1 = optr[o + 1];
    for (; k + 7 * GR_Z < k1; k += 8 * GR_Z) {
      double p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] = partial[(size_t)oslot[k + u * GR_Z] * m + a];
#pragma unroll
      for (int u = 0; u < 8; ++u) s = df_add(s, df_from_double(p[u]));
    }
    for (; k < k1; k += GR_Z) s = df_add(s, df_from_double(partial[(size_t)oslot[k] * m + a]));
  }
  red[z][x] = s;
  __syncthreads();
  if (z == 0 && a < m)
    out[(size_t)a * sa + (size_t)o * so] =
        scale * df_to_double(df_add(df_add(df_add(red[0][x], red[1][x]), red[2][x]), red[3][x]));
}

// -Mbar = L L^T by a blocked right-looking Cholesky (block CB = 32), and
// L^-1.  On this part a warp's FP64 instruction holds an SM sub-partition's
// FP64 unit for about 64 cycles whatever its active lanes, so the kernels
// keep the sequential pivot chain short and spread the products over many
// CTAs:
//   k_chol_init   A = -(M + M^T)/2 (lower triangle; zeros above)
//   per block column kb:
//     k_chol_diag   one CTA: L_kk = chol(A_kk) and Y_kk = L_kk^-1
//     k_chol_trsm   rows below: L_ik = A_ik L_kk^-T = A_ik Y_kk^T
//     k_chol_syrk   trailing lower triangle: A_ij -= L_ik L_jk^T
//   k_linv_init   diagonal blocks of L^-1 from the Y_kk
//   k_inv_pairs   L^-1 by doubling: for s = 32, 64, ..., each diagonal pair
//                 [[P, 0], [B, Q]] with known P^-1, Q^-1 has the off-diagonal
//                 block -Q^-1 B P^-1 (two batched products per level).
// A non-positive pivot sets SEA_FLAG_NOT_PD and the later kernels return.
#define CB 32
__global__ void k_chol_init(const double* __restrict__ M, int n, double* __restrict__ A) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  A[q] = (j <= i) ? -0.5 * (M[(size_t)i * n + j] + M[(size_t)j * n + i]) : 0.0;
}

// Warp w holds column w of the block (lane = row).  Step k: every column
// w > k subtracts L(:, k) L(w, k); column k + 1 is then complete and its
// warp takes the pivot at once, while the other warps still update.
__global__ void __launch_bounds__(1024)
    k_chol_diag(double* __restrict__ A, int n, int kb, unsigned* __restrict__ status,
                double* __restrict__ Y) {
  if (*status & SEA_FLAG_NOT_PD) return;
  __shared__ double Lc[CB][CB + 1];  // Lc[k][i] = L(i, k), column k final
  __shared__ double Sc[CB][CB + 1];  // Sc[k][i] = L(i, k) / L(k, k) for i > k, else 0
  __shared__ double rinv[CB];        // 1 / L(k, k)
  __shared__ int bad;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = min(CB, n - kb);
  double a = 0.0;
  if (w < nb) {
    if (lane < nb && lane >= w) a = A[(size_t)(kb + lane) * n + kb + w];
  } else if (lane == w) {
    a = 1.0;  // identity beyond the matrix edge
  }
  if (threadIdx.x == 0) bad = 0;
  auto pivot = [&]() {
    const double d = __shfl_sync(0xffffffffu, a, w);
    const bool ok = d > 0.0;
    const double r = ok ? rsqrt(d) : 0.0;
    const double l = (lane == w) ? d * r : (lane > w ? a * r : 0.0);
    Lc[w][lane] = l;
    Sc[w][lane] = (lane > w) ? l * r : 0.0;
    if (lane == 0) {
      rinv[w] = r;
      if (!ok) bad = 1;
    }
  };
  if (w == 0) pivot();
  __syncthreads();
  for (int k = 0; k < CB - 1; ++k) {
    if (bad) break;
    if (w > k) {
      a = fma(-Lc[k][lane], Lc[k][w], a);
      if (w == k + 1) pivot();
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(status, SEA_FLAG_NOT_PD);
    return;
  }
  if (w < nb && lane < nb && lane >= w) A[(size_t)(kb + lane) * n + kb + w] = Lc[w][lane];
  // column w of Y: forward substitution, t_i -= (L(i, j) / L(j, j)) t_j
  double t = (lane == w) ? 1.0 : 0.0;
  for (int j = w; j < CB - 1; ++j) t = fma(-Sc[j][lane], __shfl_sync(0xffffffffu, t, j), t);
  Y[lane * CB + w] = t * rinv[lane];
}

// Rows [kb + CB, n) of the panel, 16 per CTA (thread = row, column):
// L(i, j) = sum_{l <= j} A(i, l) Y(j, l), written in place.
__global__ void __launch_bounds__(512)
    k_chol_trsm(double* __restrict__ A, int n, int kb, const unsigned* __restrict__ status,
                const double* __restrict__ Y) {
  if (*status & SEA_FLAG_NOT_PD) return;
  __shared__ double As[16][CB + 1], Ys[CB][CB + 1];
  const int r = threadIdx.x / CB, j = threadIdx.x % CB;
  const int i = kb + CB + blockIdx.x * 16 + r;
  Ys[r][j] = Y[r * CB + j];
  Ys[r + 16][j] = Y[(r + 16) * CB + j];
  As[r][j] = (i < n && kb + j < n) ? A[(size_t)i * n + kb + j] : 0.0;
  __syncthreads();
  double x = 0.0;
  for (int l = 0; l <= j; ++l) x = fma(As[r][l], Ys[j][l], x);
  if (i < n && kb + j < n) A[(size_t)i * n + kb + j] = x;
}

// Trailing lower triangle after block column kb, one 16 x 16 tile per CTA
// (tiles (ti, tj), tj <= ti, numbered row by row).
__global__ void __launch_bounds__(256)
    k_chol_syrk(double* __restrict__ A, int n, int kb, const unsigned* __restrict__ status) {
  if (*status & SEA_FLAG_NOT_PD) return;
  int ti = 0, rem = blockIdx.x;
  while (rem > ti) {
    rem -= ti + 1;
    ++ti;
  }
  const int tj = rem;
  const int t0 = kb + CB;
  __shared__ double Li[16][CB + 1], Lj[16][CB + 1];
  const int i0 = t0 + ti * 16, j0 = t0 + tj * 16;
  for (int q = threadIdx.x; q < 16 * CB; q += blockDim.x) {
    const int r = q / CB, k = q % CB;
    const bool kin = kb + k < n;
    Li[r][k] = (i0 + r < n && kin) ? A[(size_t)(i0 + r) * n + kb + k] : 0.0;
    Lj[r][k] = (j0 + r < n && kin) ? A[(size_t)(j0 + r) * n + kb + k] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x / 16, cidx = threadIdx.x % 16;
  const int i = i0 + r, j = j0 + cidx;
  if (i >= n || j > i) return;
  double s = A[(size_t)i * n + j];
#pragma unroll 8
  for (int k = 0; k < CB; ++k) s = fma(-Li[r][k], Lj[cidx][k], s);
  A[(size_t)i * n + j] = s;
}

// Linv = block diagonal of the Y_kk (zeros elsewhere).
__global__ void k_linv_init(const double* __restrict__ Y, int n, double* __restrict__ Linv) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  const int b = i / CB;
  Linv[q] = (j / CB == b && j <= i) ? Y[(size_t)b * CB * CB + (i % CB) * CB + (j % CB)] : 0.0;
}

// One level of the doubling.  Pair p covers rows/columns [o, o + s + s2),
// o = 2 s p, s2 = min(s, n - o - s): P = Linv[o.., o..] (s x s), B = L[o+s..,
// o..] (s2 x s), Q = Linv[o+s.., o+s..] (s2 x s2), all known.  phase 0:
// T_p = B P (P lower: k >= j);  phase 1: Linv[o+s+i][o+j] = -(Q T_p)[i][j]
// (Q lower: k <= i).  16 x 16 output tile per CTA, grid (s/16, s/16, pairs).
__global__ void __launch_bounds__(256)
    k_inv_pairs(int n, int s, int phase, const double* __restrict__ L, double* __restrict__ Linv,
                double* __restrict__ T) {
  const int p = blockIdx.z, o = 2 * s * p;
  const int s2 = min(s, n - o - s);
  if (s2 <= 0) return;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  if (i0 >= s2) return;
  const int i = i0 + ty, j = j0 + tx;
  double* Tp = T + (size_t)p * s * s;  // [s2][s]
  __shared__ double As[16][17], Bs[16][17];
  double acc = 0.0;
  // phase 0: k in [j0, s); phase 1: k in [0, min(i0 + 16, s2))
  const int kbeg = phase == 0 ? j0 : 0;
  const int kend = phase == 0 ? s : min(i0 + 16, s2);
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    const int ka = k0 + tx, kr = k0 + ty;
    double av = 0.0, bv = 0.0;
    if (phase == 0) {
      if (i < s2 && ka < s) av = L[(size_t)(o + s + i) * n + o + ka];
      if (kr < s && j < s) bv = Linv[(size_t)(o + kr) * n + o + j];
    } else {
      if (i < s2 && ka < s2) av = Linv[(size_t)(o + s + i) * n + o + s + ka];
      if (kr < s2 && j < s) bv = Tp[(size_t)kr * s + j];
    }
    As[ty][tx] = av;
    Bs[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (i >= s2 || j >= s) return;
  if (phase == 0)
    Tp[(size_t)i * s + j] = acc;
  else
    Linv[(size_t)(o + s + i) * n + o + j] = -acc;
}

// ---------------------------------------------------------------------------
// Eigen-decomposition form of the ACE build (App. A): -Mbar = Q Lambda Q^T
// by the cyclic Jacobi method with round-robin ordering (each round rotates
// ne/2 disjoint index pairs at once; ne = n rounded up to even).  Per round,
// k_jac_rows computes each pair's rotation from the current matrix and
// rotates its two rows; k_jac_cols rotates the two columns of S and of Q.
// App. A's zeta_k = -D Q Lambda^-1/2 is complex where lambda_k < 0; with the
// Hermitian inner product <zeta_k| of the plane-wave code the phase cancels
// and V^ACE = -sum_k |zeta_k><zeta_k| = -W Q |Lambda|^-1 Q^T W^T (reading;
// the same as the Cholesky form when -Mbar is positive definite).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void jac_pair(int k, int r, int ne, int* p, int* q) {
  // positions k and ne-1-k of the circle: position 0 holds index 0, position
  // i >= 1 holds 1 + (i - 1 + r) mod (ne - 1)
  auto idx = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (ne - 1); };
  *p = idx(k);
  *q = idx(ne - 1 - k);
}

__global__ void k_jac_init(const double* __restrict__ M, int n, double* __restrict__ S,
                           double* __restrict__ Q) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  S[t] = -0.5 * (M[(size_t)i * n + j] + M[(size_t)j * n + i]);
  Q[t] = (i == j) ? 1.0 : 0.0;
}

__global__ void k_jac_rows(double* __restrict__ S, int n, int ne, int r, double* __restrict__ cs) {
  int p, q;
  jac_pair(blockIdx.x, r, ne, &p, &q);
  __shared__ double sc[2];
  if (threadIdx.x == 0) {
    double c = 1.0, s = 0.0;
    if (p < n && q < n) {
      const double apq = S[(size_t)p * n + q];
      if (apq != 0.0) {
        const double th = (S[(size_t)q * n + q] - S[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        c = 1.0 / sqrt(t * t + 1.0);
        s = t * c;
      }
    }
    sc[0] = c;
    sc[1] = s;
    cs[2 * blockIdx.x] = c;
    cs[2 * blockIdx.x + 1] = s;
  }
  __syncthreads();
  if (p >= n || q >= n) return;
  const double c = sc[0], s = sc[1];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = S[(size_t)p * n + j], b = S[(size_t)q * n + j];
    S[(size_t)p * n + j] = c * a - s * b;
    S[(size_t)q * n + j] = s * a + c * b;
  }
}

__global__ void k_jac_cols(double* __restrict__ S, double* __restrict__ Q, int n, int ne, int r,
                           const double* __restrict__ cs) {
  int p, q;
  jac_pair(blockIdx.x, r, ne, &p, &q);
  if (p >= n || q >= n) return;
  const double c = cs[2 * blockIdx.x], s = cs[2 * blockIdx.x + 1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = S[(size_t)i * n + p], b = S[(size_t)i * n + q];
    S[(size_t)i * n + p] = c * a - s * b;
    S[(size_t)i * n + q] = s * a + c * b;
    a = Q[(size_t)i * n + p];
    b = Q[(size_t)i * n + q];
    Q[(size_t)i * n + p] = c * a - s * b;
    Q[(size_t)i * n + q] = s * a + c * b;
  }
}

// out[0] = sum of squared off-diagonal entries, out[1] = sum of squared
// diagonal entries (fixed-order block reduction).
__global__ void k_jac_norms(const double* __restrict__ S, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double off = 0.0, dia = 0.0;
  for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {
    const double v = S[t];
    if ((int)(t / n) == (int)(t % n))
      dia = fma(v, v, dia);
    else
      off = fma(v, v, off);
  }
  off = block_sum(off, red);
  __syncthreads();
  dia = block_sum(dia, red);
  if (threadIdx.x == 0) {
    out[0] = off;
    out[1] = dia;
  }
}

// inv[i] = 1/|lambda_i| for |lambda_i| > cut, else 0 (eigenvalues within
// 1e-13 max|lambda| of zero are dropped); counts negative and dropped
// eigenvalues.
__global__ void k_jac_invdiag(const double* __restrict__ S, int n, double* __restrict__ inv,
                              int* __restrict__ counts) {
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(S[(size_t)i * n + i]));
    mx = m;
  }
  __syncthreads();
  const double cut = 1e-13 * mx;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double l = S[(size_t)i * n + i];
    inv[i] = fabs(l) > cut ? 1.0 / fabs(l) : 0.0;
    if (l < -cut) atomicAdd(&counts[0], 1);
    if (!(fabs(l) > cut)) atomicAdd(&counts[1], 1);
  }
}

// B[i][v] *= d[i]
__global__ void k_scale_rows(double* __restrict__ B, const double* __restrict__ d, int n, int m) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * m) return;
  B[t] *= d[t / m];
}

// C[n1][n2] = op(A) B, op(A)(i, k) = A[k][i] if transA else A[i][k]; A is
// n1 x n1 (square), B is [n1][n2].  16 x 16 shared-memory tiles.  With
// `lower`, A's zero upper triangle is not multiplied.
__global__ void k_small_gemm(const double* __restrict__ A, int transA, const double* __restrict__ B,
                             int n1, int n2, double* __restrict__ C, int lower) {
  __shared__ double As[16][17], Bs[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  // lower: A is lower triangular (zeros above the diagonal, exactly), so
  // op(A)(i, k) vanishes for k > i (A B) or k < i (A^T B); those tiles are
  // skipped (their products would add exact zeros)
  const int kbeg = (lower && transA) ? blockIdx.y * 16 : 0;
  const int kend = (lower && !transA) ? min(n1, (int)(blockIdx.y + 1) * 16) : n1;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    double av = 0.0;
    if (i < n1 && ka < n1) av = transA ? A[(size_t)ka * n1 + i] : A[(size_t)i * n1 + ka];
    As[threadIdx.y][threadIdx.x] = av;
    Bs[threadIdx.y][threadIdx.x] = (kb < n1 && j < n2) ? B[(size_t)kb * n2 + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (i < n1 && j < n2) C[(size_t)i * n2 + j] = acc;
}

// The same product in double-float arithmetic for the mixed form (FP64
// operands split exactly into FP32 pairs to about 2^-47, FP32 pipes instead
// of the FP64 unit, one rounding to FP64 at the end).
__global__ void __launch_bounds__(256)
    k_small_gemm_df(const double* __restrict__ A, int transA, const double* __restrict__ B,
                    int n1, int n2, double* __restrict__ C, int lower) {
  __shared__ float Ah[16][17], Al[16][17], Bh[16][17], Bl[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  DF acc{0.f, 0.f};
  const int kbeg = (lower && transA) ? blockIdx.y * 16 : 0;
  const int kend = (lower && !transA) ? min(n1, (int)(blockIdx.y + 1) * 16) : n1;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    double av = 0.0;
    if (i < n1 && ka < n1) av = transA ? A[(size_t)ka * n1 + i] : A[(size_t)i * n1 + ka];
    const double bv = (kb < n1 && j < n2) ? B[(size_t)kb * n2 + j] : 0.0;
    const float2 as = split64(av), bs = split64(bv);
    Ah[threadIdx.y][threadIdx.x] = as.x;
    Al[threadIdx.y][threadIdx.x] = as.y;
    Bh[threadIdx.y][threadIdx.x] = bs.x;
    Bl[threadIdx.y][threadIdx.x] = bs.y;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k)
      acc = df_fma(DF{Ah[threadIdx.y][k], Al[threadIdx.y][k]}, DF{Bh[k][threadIdx.x], Bl[k][threadIdx.x]},
                   acc);
    __syncthreads();
  }
  if (i < n1 && j < n2) C[(size_t)i * n2 + j] = df_to_double(acc);
}

// out[v][r] = sign * sum_{j in tile list} W[j][r] H(j, v), H(j, v) =
// H[j * hj + v * hv], for every point r of the tile and v in a chunk of 32:
// thread = (point, half of the chunk), 16 accumulators.
#define EV 32
__global__ void __launch_bounds__(256)
    k_tile_expand(const double* __restrict__ W, TileGeom G, size_t ng,
                  const int* __restrict__ tptr, const int* __restrict__ tlist,
                  const int* __restrict__ tsub, const double* __restrict__ H, long long hj,
                  long long hv, int m, double sign, double* __restrict__ out) {
  const int T = blockIdx.x;
  const int v0 = blockIdx.y * EV;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  extern __shared__ double Hs[];  // [nJ][EV]
  for (int idx = threadIdx.x; idx < nJ * EV; idx += blockDim.x) {
    const int jl = idx / EV, vl = idx % EV;
    Hs[idx] = (v0 + vl < m) ? H[(long long)tlist[j0 + jl] * hj + (long long)(v0 + vl) * hv] : 0.0;
  }
  __syncthreads();
  const int pt = threadIdx.x % TP, vh = threadIdx.x / TP;
  const long long g = tile_point(G, T, pt);
  double acc[EV / 2];
#pragma unroll
  for (int u = 0; u < EV / 2; ++u) acc[u] = 0.0;
  const int pz = pt / (TX * TY), py = (pt / TX) % TY, px = pt % TX;  // pz: one per warp
  for (int jl = 0; jl < nJ; ++jl) {
    const int sb = tsub[j0 + jl];
    if (pz < ((sb >> 16) & 15) || pz >= ((sb >> 20) & 15)) continue;  // warp-uniform
    const bool in = px >= (sb & 15) && px < ((sb >> 4) & 15) && py >= ((sb >> 8) & 15) &&
                    py < ((sb >> 12) & 15);
    const double w = (g >= 0 && in) ? W[(size_t)tlist[j0 + jl] * ng + g] : 0.0;
    const double* hrow = Hs + jl * EV + vh * (EV / 2);
#pragma unroll
    for (int u = 0; u < EV / 2; ++u) acc[u] = fma(w, hrow[u], acc[u]);
  }
  if (g < 0) return;
#pragma unroll
  for (int u = 0; u < EV / 2; ++u) {
    const int v = v0 + vh * (EV / 2) + u;
    if (v < m) out[(size_t)v * ng + g] = sign * acc[u];
  }
}


// E_xx^ACE = sum_i <phi_i|V^ACE|phi_i> (Eq. exx_ace).  With G = W^T Phi dV
// = M^T, V^ACE phi_i = -W K G_i and so E = -tr(M K M^T); K = L^-T L^-1 for the
// Cholesky form, Q |Lambda|^-1 Q^T for the eigen form.  Written as
//   E = -sum_k d_k sum_i Y[k][i]^2,  Y[k][i] = sum_j A(k, j) M[i][j],
// with A = L^-1, d = 1 (then Y[k][i] = <phi_i|xi_k>, the second form of
// Eq. exx_ace), or A(k, j) = Q[j][k], d_k = 1/|lambda_k| (0 where dropped).
// Warp w forms Y[k][i] for one block of 32 rows i (lane = i) and the two
// rows k = kp and n - 1 - kp, so that with the triangular A = L^-1 (A(k, j)
// = 0 for j > k, not read) every warp does n + 1 multiply-adds; A's entries
// are the same for the warp's lanes (one broadcast load), each lane walks
// its own row of M.  The warp's sum of d_k Y^2 (lane order, then a fixed
// butterfly) goes to part[w]; k_exx_ace_sum adds the parts in order.
__global__ void __launch_bounds__(64)
    k_exx_ace_rows(const double* __restrict__ M, const double* __restrict__ A, int transA,
                   const double* __restrict__ d, int n, double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 2 + (threadIdx.x >> 5);
  const int nib = (n + 31) / 32, npair = (n + 1) / 2;
  if (gw >= nib * npair) return;
  const int ib = gw % nib, kp = gw / nib;
  const int i = ib * 32 + lane, k1 = kp, k2 = n - 1 - kp;
  const bool tri = !transA;
  const double* mi = M + (size_t)(i < n ? i : 0) * n;
  auto a_at = [&](int k, int j) { return transA ? A[(size_t)j * n + k] : A[(size_t)k * n + j]; };
  double y1 = 0.0, y2 = 0.0;
  const int jboth = tri ? k1 + 1 : n, jend = tri ? k2 + 1 : n;
  for (int j = 0; j < jboth; ++j) {
    const double mv = mi[j];
    y1 = fma(a_at(k1, j), mv, y1);
    y2 = fma(a_at(k2, j), mv, y2);
  }
  for (int j = jboth; j < jend; ++j) y2 = fma(a_at(k2, j), mi[j], y2);
  double s = 0.0;
  if (i < n) {
    s = (d ? d[k1] : 1.0) * y1 * y1;
    if (k2 != k1) s = fma((d ? d[k2] : 1.0) * y2, y2, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[gw] = s;
}

// out = -sum_w part[w] (fixed order: thread strides, then the block sum).
__global__ void k_exx_ace_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) t += part[k];
  t = block_sum(t, red);
  if (threadIdx.x == 0) *out = -t;
}

static cudaError_t launch_exx_ace(sea_ctx* c, int transA, const double* d) {
  const int n = c->n_orb;
  const int nparts = ((n + 31) / 32) * ((n + 1) / 2);
  if (!sea_ensure(c, c->Gbuf, (size_t)nparts * sizeof(double))) return cudaErrorMemoryAllocation;
  double* part = (double*)c->Gbuf.p;
  k_exx_ace_rows<<<(nparts + 1) / 2, 64, 0, c->stream>>>(
      (const double*)c->Mbuf.p, (const double*)c->Linv.p, transA, d, n, part);
  k_exx_ace_sum<<<1, 256, 0, c->stream>>>(part, nparts, (double*)c->exx_dev.p + SEA_EXX_ACE_SLOT);
  c->launches += 2;
  return cudaGetLastError();
}

// The contractions with W: FP64 kernels for the plain form, the
// tensor-core kernel (exact BF16 digit splitting) for the mixed form.
static cudaError_t launch_gram(sea_ctx* c, const double* A, int m, const TileGeom& G,
                               const int* tptr, const int* tlist, const int* tsub) {
  const double* W = (const double*)c->vxx_dev.p;
  if (c->prm.precision == 1)
    return launch_gram_tc(c->stream, c->device, A, m, G, c->ng, c->n_tiles, tptr, c->tile_inc,
                          c->wdig.p, (double*)c->partial.p, (int*)c->counts.p + 20,
                          (unsigned*)c->status.p);
  k_gram_partial<<<dim3(c->n_tiles, (m + GA - 1) / GA), 256, GRAM_SMEM, c->stream>>>(
      A, m, W, G, c->ng, tptr, tlist, tsub, (double*)c->partial.p);
  return cudaGetLastError();
}

static cudaError_t launch_expand(sea_ctx* c, const TileGeom& G, const int* tptr,
                                 const int* tlist, const int* tsub, const double* H, long long hj,
                                 long long hv, int m, double sign, double* out) {
  if (c->prm.precision == 1) {
    // tiles with at most expand_tc_max_list() W rows on the tensor cores,
    // longer lists (if any) by the FP32 kernel
    if (!sea_ensure(c, c->xevb, (size_t)max(c->n_tiles, 1) * m * sizeof(int)))
      return cudaErrorMemoryAllocation;
    const cudaError_t e = launch_expand_tc(c->stream, c->device, c->wx.p, G, c->ng, c->n_tiles,
                                           tptr, tlist, H, hj, hv, m, sign < 0.0, out,
                                           (int*)c->xevb.p, (int*)c->counts.p + 24,
                                           (unsigned*)c->status.p);
    if (e != cudaSuccess) return e;
    if (c->max_tile_list > expand_tc_max_list()) {
      const size_t smem = (size_t)c->max_tile_list * 32 * sizeof(float2);
      k_tile_expand_x<<<dim3(c->n_tiles, (m + 31) / 32), 256, smem, c->stream>>>(
          (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist, tsub, H, hj, hv, m, sign,
          expand_tc_max_list(), out);
      c->launches += 1;
    }
  } else {
    const size_t smem = (size_t)c->max_tile_list * EV * sizeof(double);
    k_tile_expand<<<dim3(c->n_tiles, (m + EV - 1) / EV), 256, smem, c->stream>>>(
        (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist, tsub, H, hj, hv, m, sign, out);
  }
  return cudaGetLastError();
}

// Scratch (doubles) of the L^-1 doubling: the largest level's pairs x s x s.
static size_t inv_scratch_doubles(int n) {
  size_t m = 1;
  for (int s = CB; s < n; s *= 2) {
    const size_t pairs = (size_t)((n - s + 2 * s - 1) / (2 * s));
    m = std::max(m, pairs * s * s);
  }
  return m;
}

// The Cholesky of -Mbar, L^-1 and E_xx^ACE: about 30 small launches whose
// shapes depend on n alone, replayed from a graph (run_graph; recorded again
// when a buffer moves or n or the form changes).
static cudaError_t enqueue_chol_chain(sea_ctx* c) {
  const int n = c->n_orb;
  if (c->prm.precision == 1) {  // one cooperative launch of block tasks, double-float
    c->launches += 1;
    return launch_chol_flow(c->stream, c->device, (const double*)c->Mbuf.p, n,
                            (double*)c->Lbuf.p, (double*)c->Linv.p, c->flowbuf.p,
                            (unsigned*)c->status.p, (double*)c->exx_dev.p + SEA_EXX_ACE_SLOT);
  }
  k_chol_init<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, c->stream>>>(
      (const double*)c->Mbuf.p, n, (double*)c->Lbuf.p);
  double* L = (double*)c->Lbuf.p;
  double* Y = (double*)c->Abuf.p;  // Y_kk blocks, CB x CB each
  unsigned* status = (unsigned*)c->status.p;
  int nchol = 1;
  for (int kb = 0, b = 0; kb < n; kb += CB, ++b) {
    k_chol_diag<<<1, 1024, 0, c->stream>>>(L, n, kb, status, Y + (size_t)b * CB * CB);
    const int rows = n - kb - CB;
    if (rows > 0) {
      const int nt = (rows + 15) / 16;
      k_chol_trsm<<<nt, 512, 0, c->stream>>>(L, n, kb, status, Y + (size_t)b * CB * CB);
      k_chol_syrk<<<nt * (nt + 1) / 2, 256, 0, c->stream>>>(L, n, kb, status);
      nchol += 2;
    }
    nchol += 1;
  }
  double* Linv = (double*)c->Linv.p;
  k_linv_init<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, c->stream>>>(Y, n, Linv);
  for (int s = CB; s < n; s *= 2) {
    const int pairs = (n - s + 2 * s - 1) / (2 * s);
    const dim3 g((s + 15) / 16, (s + 15) / 16, pairs);
    double* T = (double*)c->Hbuf2.p;
    k_inv_pairs<<<g, 256, 0, c->stream>>>(n, s, 0, L, Linv, T);
    k_inv_pairs<<<g, 256, 0, c->stream>>>(n, s, 1, L, Linv, T);
    nchol += 2;
  }
  c->launches += 8 + nchol;
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_exx_ace(c, 0, nullptr);  // Y = L^-1 M^T
}

static cudaError_t launch_chol_chain(sea_ctx* c) {
  const int n = c->n_orb;
  const int nparts = ((n + 31) / 32) * ((n + 1) / 2);
  if (!sea_ensure(c, c->Gbuf, (size_t)nparts * sizeof(double))) return cudaErrorMemoryAllocation;
  if (c->prm.precision == 1 && !sea_ensure(c, c->flowbuf, chol_flow_bytes(n)))
    return cudaErrorMemoryAllocation;
  const std::vector<uintptr_t> sig = {
      (uintptr_t)n, (uintptr_t)c->prm.precision, (uintptr_t)c->Mbuf.p, (uintptr_t)c->Lbuf.p,
      (uintptr_t)c->Abuf.p, (uintptr_t)c->Linv.p, (uintptr_t)c->Hbuf2.p, (uintptr_t)c->Gbuf.p,
      (uintptr_t)c->status.p, (uintptr_t)c->exx_dev.p, (uintptr_t)c->flowbuf.p};
  return run_graph(c, c->g_chol, sig, [&]() { return enqueue_chol_chain(c); });
}

// The tile-major and orbital-major lists of W's support on stream st: the
// (orbital, tile) incidences, per-tile counts and their scan, the lists.
// The list arrays are sized for every (orbital, tile) pair (list_cap), so no
// count has to reach the host before the lists are formed; the incidence
// count and the longest tile list land in counts[10] and counts[12].
cudaError_t launch_ace_lists(sea_ctx* c, cudaStream_t st) {
  const int n = c->n_orb;
  const TileGeom G = make_tile_geom(c->N);
  const int nt = G.ntx * G.nty * G.ntz;
  const long long ninc = (long long)n * nt;
  const long long cap = std::max(ninc, 1LL);
  if (!sea_ensure(c, c->tmask, ninc * sizeof(int) * 3) ||
      !sea_ensure(c, c->tptr_t, (size_t)(nt + 1) * sizeof(int) * 2) ||
      !sea_ensure(c, c->tptr_o, (size_t)(n + 1) * sizeof(int) * 2) ||
      !sea_ensure(c, c->tlist_t, (size_t)cap * sizeof(int) * 2) ||
      !sea_ensure(c, c->tlist_o, (size_t)cap * sizeof(int) * 2))
    return cudaErrorMemoryAllocation;
  c->n_tiles = nt;
  c->list_cap = cap;
  int* inc = (int*)c->tmask.p;
  int* gidx = inc + ninc;
  int* sub = inc + 2 * ninc;
  int* tcnt = (int*)c->tptr_t.p;
  int* tptr = tcnt + (nt + 1);
  int* ocnt = (int*)c->tptr_o.p;
  int* optr = ocnt + (n + 1);
  int* counts = (int*)c->counts.p;
  int* tlist = (int*)c->tlist_t.p;
  int* tsub = tlist + cap;
  int* olist = (int*)c->tlist_o.p;
  int* oslot = olist + cap;
  k_tile_incidence<<<(unsigned)((ninc + 255) / 256), 256, 0, st>>>(
      (const Entry*)c->ewin.p, (const int*)c->eptr.p, n, G, nt, c->w_dense ? 1 : 0, inc, sub);
  k_tile_lists<<<(nt + 7) / 8, 256, 0, st>>>(inc, sub, n, nt, 0, tcnt, nullptr, nullptr, nullptr,
                                             nullptr);
  k_scan_small<<<1, 1024, 0, st>>>(tcnt, nt, tptr, counts + 10);
  k_max_int<<<1, 1024, 0, st>>>(tcnt, nt, counts + 12);
  k_tile_lists<<<(nt + 7) / 8, 256, 0, st>>>(inc, sub, n, nt, 1, nullptr, tptr, tlist, tsub, gidx);
  k_orb_lists<<<(n * 32 + 127) / 128, 128, 0, st>>>(gidx, n, nt, 0, ocnt, nullptr, nullptr,
                                                    nullptr);
  k_scan_small<<<1, 1024, 0, st>>>(ocnt, n, optr, counts + 11);
  k_orb_lists<<<(n * 32 + 127) / 128, 128, 0, st>>>(gidx, n, nt, 1, nullptr, optr, olist, oslot);
  c->launches += 8;
  return cudaGetLastError();
}

// M, Cholesky and L^-1 (and the tile lists first, unless sea_apply_vxx
// formed them with its plan: then their counts are already on the host).
cudaError_t launch_ace_build(sea_ctx* c) {
  const int n = c->n_orb;
  const TileGeom G = make_tile_geom(c->N);
  if (!sea_ensure(c, c->Mbuf, (size_t)n * n * sizeof(double)) ||
      !sea_ensure(c, c->Lbuf, (size_t)n * n * sizeof(double)) ||
      !sea_ensure(c, c->Linv, (size_t)n * n * sizeof(double)) ||
      !sea_ensure(c, c->Abuf, (size_t)((n + CB - 1) / CB) * CB * CB * sizeof(double)) ||
      !sea_ensure(c, c->Hbuf2, inv_scratch_doubles(n) * sizeof(double)))
    return cudaErrorMemoryAllocation;
  cudaError_t err = cudaSuccess;
  if (c->w_dense || !c->lists_ready) {
    c->lists_ready = false;
    err = launch_ace_lists(c, c->stream);
    if (err != cudaSuccess) return err;
    int hc[3] = {0, 0, 0};
    cudaMemcpyAsync(hc, (int*)c->counts.p + 10, sizeof(hc), cudaMemcpyDeviceToHost, c->stream);
    err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) return err;
    c->tile_inc = hc[0];
    c->max_tile_list = hc[2];
  }
  const int nt = c->n_tiles;
  const int hinc = c->tile_inc;
  {
    const size_t smem = (size_t)c->max_tile_list * EV * sizeof(double);
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(k_tile_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_tile_expand_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
      if (err != cudaSuccess) return err;
    }
  }
  if (!sea_ensure(c, c->partial, (size_t)max(hinc, 1) * n * sizeof(double)))
    return cudaErrorMemoryAllocation;
  const int* tptr = (const int*)c->tptr_t.p + (nt + 1);
  const int* optr = (const int*)c->tptr_o.p + (n + 1);
  const int* tlist = (const int*)c->tlist_t.p;
  const int* tsub = tlist + c->list_cap;
  const int* oslot = (const int*)c->tlist_o.p + c->list_cap;
  // M = Phi^T W dV
  err = cudaFuncSetAttribute(k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GRAM_SMEM);
  if (err != cudaSuccess) return err;
  if (c->prm.precision == 1) {  // W's digits for the tensor-core contractions
    if (!sea_ensure(c, c->wdig, w_digits_bytes(hinc))) return cudaErrorMemoryAllocation;
    err = launch_w_digits(c->stream, (const double*)c->vxx_dev.p, G, c->ng, nt, c->max_tile_list,
                          tptr, tlist, hinc, c->wdig.p);
    if (err != cudaSuccess) return err;
    if (!sea_ensure(c, c->wx, wx_digits_bytes(nt, hinc))) return cudaErrorMemoryAllocation;
    c->launches += 2;
  }
  cudaEventRecord(c->ev[10], c->stream);
  err = launch_gram(c, (const double*)c->phi.p, n, G, tptr, tlist, tsub);
  if (err != cudaSuccess) return err;
  cudaEventRecord(c->ev[11], c->stream);
  if (c->prm.precision == 1) {
    // W's per-tile images for the expansion (used by sea_apply_ace only) on
    // a second stream, beside the latency-bound Cholesky chain below; the
    // context stream waits for them before the build ends
    err = cudaStreamWaitEvent(c->xfer[0], c->ev[11], 0);
    if (err == cudaSuccess)
      err = launch_wx_digits(c->xfer[0], (const double*)c->vxx_dev.p, G, c->ng, nt, tptr, tlist,
                             tsub, c->wx.p);
    if (err == cudaSuccess) err = cudaEventRecord(c->xev[0], c->xfer[0]);
    if (err != cudaSuccess) return err;
  }
  (c->prm.precision == 1 ? k_gram_reduce_df : k_gram_reduce)<<<dim3((n + GR_A - 1) / GR_A, n), GR_A * GR_Z, 0, c->stream>>>(
      (const double*)c->partial.p, n, n, optr, oslot, c->dV, (double*)c->Mbuf.p,
      n, 1);
  c->launches += 2;
  err = launch_chol_chain(c);
  if (err == cudaSuccess && c->prm.precision == 1) err = cudaStreamWaitEvent(c->stream, c->xev[0], 0);
  return err;
}

// Eigen form (App. A) after M is known: Q into Linv, S (eigenvalues on the
// diagonal) into Lbuf, 1/lambda into Abuf.  Host loop over sweeps; stops when
// the off-diagonal mass is below 1e-30 of the diagonal mass (or 60 sweeps).
cudaError_t launch_ace_eigen(sea_ctx* c) {
  const int n = c->n_orb;
  const int ne = n + (n & 1);
  if (!sea_ensure(c, c->Gbuf, (size_t)max(ne, 2) * sizeof(double) * 2 + 64) ||
      !sea_ensure(c, c->Abuf, (size_t)n * CB * sizeof(double) + (size_t)n * sizeof(double)))
    return cudaErrorMemoryAllocation;
  double* S = (double*)c->Lbuf.p;
  double* Q = (double*)c->Linv.p;
  double* cs = (double*)c->Gbuf.p;
  double* norms = cs + 2 * max(ne, 2);
  int* counts = (int*)c->counts.p + 14;
  k_jac_init<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, c->stream>>>(
      (const double*)c->Mbuf.p, n, S, Q);
  c->launches += 1;
  int sweeps = 0;
  for (; sweeps < 60 && ne >= 2; ++sweeps) {
    double hn[2] = {0.0, 0.0};
    k_jac_norms<<<1, 1024, 0, c->stream>>>(S, n, norms);
    cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    c->launches += 1;
    if (!(hn[0] > 1e-30 * hn[1])) break;
    for (int r = 0; r < ne - 1; ++r) {
      k_jac_rows<<<ne / 2, 128, 0, c->stream>>>(S, n, ne, r, cs);
      k_jac_cols<<<ne / 2, 128, 0, c->stream>>>(S, Q, n, ne, r, cs);
    }
    c->launches += 2 * (ne - 1);
  }
  cudaMemsetAsync(counts, 0, 2 * sizeof(int), c->stream);
  k_jac_invdiag<<<1, 256, 0, c->stream>>>(S, n, (double*)c->Abuf.p, counts);
  c->launches += 1;
  int hc[2] = {0, 0};
  cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  c->stats.ace_eigen_sweeps = sweeps;
  c->stats.ace_negative_eigenvalues = hc[0];
  c->stats.ace_dropped_eigenvalues = hc[1];
  c->ace_eigen = true;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_exx_ace(c, 1, (const double*)c->Abuf.p);  // Y = Q^T M^T, d = 1/|lambda|
}

cudaError_t launch_ace_apply(sea_ctx* c, const double* psi, int nv, double* out) {
  const int n = c->n_orb;
  const TileGeom G = make_tile_geom(c->N);
  const int nt = c->n_tiles;
  const int hinc = c->tile_inc;
  if (!sea_ensure(c, c->partial,
                  (size_t)max(hinc, 1) * max(n, nv) * sizeof(double)) ||
      !sea_ensure(c, c->Gbuf, (size_t)n * nv * sizeof(double)) ||
      !sea_ensure(c, c->Hbuf, (size_t)n * nv * sizeof(double)) ||
      !sea_ensure(c, c->Hbuf2, (size_t)n * nv * sizeof(double)))
    return cudaErrorMemoryAllocation;
  const int* tptr = (const int*)c->tptr_t.p + (nt + 1);
  const int* tlist = (const int*)c->tlist_t.p;
  const int* tsub = tlist + c->list_cap;
  const int* optr = (const int*)c->tptr_o.p + (n + 1);
  const int* olist = (const int*)c->tlist_o.p;
  const int* oslot = olist + c->list_cap;
  // G[o][v] = <W_o|psi_v> dV
  cudaEventRecord(c->ev[12], c->stream);
  {
    const cudaError_t e = launch_gram(c, psi, nv, G, tptr, tlist, tsub);
    if (e != cudaSuccess) return e;
  }
  cudaEventRecord(c->ev[13], c->stream);
  (c->prm.precision == 1 ? k_gram_reduce_df : k_gram_reduce)<<<dim3((nv + GR_A - 1) / GR_A, n), GR_A * GR_Z, 0, c->stream>>>(
      (const double*)c->partial.p, nv, n, optr, oslot, c->dV, (double*)c->Gbuf.p,
      1, nv);
  // H = (-Mbar)^-1 G = L^-T (L^-1 G), or Q |Lambda|^-1 Q^T G in the eigen form
  dim3 gb((nv + 15) / 16, (n + 15) / 16), tb(16, 16);
  // the mixed form's products in double-float (the FP64 unit is the bound of the FP64 ones)
  auto small_gemm = c->prm.precision == 1 ? k_small_gemm_df : k_small_gemm;
  if (c->ace_eigen) {
    small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 1, (const double*)c->Gbuf.p,
                                           n, nv, (double*)c->Hbuf2.p, 0);
    k_scale_rows<<<(unsigned)(((size_t)n * nv + 255) / 256), 256, 0, c->stream>>>(
        (double*)c->Hbuf2.p, (const double*)c->Abuf.p, n, nv);
    small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 0, (const double*)c->Hbuf2.p,
                                           n, nv, (double*)c->Hbuf.p, 0);
    c->launches += 1;
  } else {
    small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 0, (const double*)c->Gbuf.p,
                                           n, nv, (double*)c->Hbuf2.p, 1);
    small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 1, (const double*)c->Hbuf2.p,
                                           n, nv, (double*)c->Hbuf.p, 1);
  }
  // out[v] = -sum_j W_j H[j][v]
  cudaEventRecord(c->ev[14], c->stream);
  cudaError_t ex = launch_expand(c, G, tptr, tlist, tsub, (const double*)c->Hbuf.p, nv, 1, nv,
                                 -1.0, out);
  if (ex != cudaSuccess) return ex;
  cudaEventRecord(c->ev[15], c->stream);
  c->launches += 5;
  return cudaGetLastError();
}

cudaError_t launch_ace_vectors(sea_ctx* c, double* xi) {
  const int n = c->n_orb;
  const TileGeom G = make_tile_geom(c->N);
  const int nt = c->n_tiles;
  const int* tptr = (const int*)c->tptr_t.p + (nt + 1);
  const int* tlist = (const int*)c->tlist_t.p;
  const int* tsub = tlist + c->list_cap;
  // Xi[k][r] = sum_j W[j][r] (L^-1)[k][j]:  H(j, k) = Linv[k * n + j]
  cudaError_t ex = launch_expand(c, G, tptr, tlist, tsub, (const double*)c->Linv.p, 1, n, n, 1.0, xi);
  if (ex != cudaSuccess) return ex;
  c->launches += 1;
  return cudaGetLastError();
}

}  // namespace sea
