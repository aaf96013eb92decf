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

#define TX 8
#define TY 4
#define TZ 4
#define TP (TX * TY * TZ)

struct TileGeom {
  int nx, ny, nz, ntx, nty, ntz;
};

__device__ __forceinline__ bool cyc_meets(int s, int L, int a, int b, int n) {
  // cyclic [s, s+L) (s wrapped) meets [a, b) (0 <= a < b <= n)
  if (L >= n) return true;
  return (wrapi(s - a, n) < b - a) || (wrapi(a - s, n) < L);
}

// inc[o][T] = 1 if any entry window of orbital o touches tile T.
__global__ void k_tile_incidence(const Entry* __restrict__ ent, const int* __restrict__ eptr,
                                 int n_orb, TileGeom G, int n_tiles, int* __restrict__ inc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_orb * n_tiles) return;
  const int o = (int)(t / n_tiles), T = (int)(t % n_tiles);
  const int txi = T % G.ntx, tyi = (T / G.ntx) % G.nty, tzi = T / (G.ntx * G.nty);
  const int ax = txi * TX, bx = min(G.nx, ax + TX);
  const int ay = tyi * TY, by = min(G.ny, ay + TY);
  const int az = tzi * TZ, bz = min(G.nz, az + TZ);
  int hit = 0;
  for (int k = eptr[o]; k < eptr[o + 1] && !hit; ++k) {
    const Entry e = ent[k];
    hit = cyc_meets(wrapi(e.ws[0], G.nx), e.wl[0], ax, bx, G.nx) &&
          cyc_meets(wrapi(e.ws[1], G.ny), e.wl[1], ay, by, G.ny) &&
          cyc_meets(wrapi(e.ws[2], G.nz), e.wl[2], az, bz, G.nz);
  }
  inc[t] = hit;
}

// Tile-major lists: thread per tile, orbitals ascending.  mode 0 counts,
// mode 1 writes the list and the incidence index gidx[o][T].
__global__ void k_tile_lists(const int* __restrict__ inc, int n_orb, int n_tiles, int mode,
                             int* __restrict__ cnt, const int* __restrict__ ptr,
                             int* __restrict__ list, int* __restrict__ gidx) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= n_tiles) return;
  int c = 0;
  int pos = mode ? ptr[T] : 0;
  for (int o = 0; o < n_orb; ++o) {
    const size_t q = (size_t)o * n_tiles + T;
    if (!inc[q]) {
      if (mode) gidx[q] = -1;
      continue;
    }
    ++c;
    if (mode) {
      list[pos] = o;
      gidx[q] = pos;
      ++pos;
    }
  }
  if (!mode) cnt[T] = c;
}

// Orbital-major lists: thread per orbital, tiles ascending, with the
// incidence index of each (orbital, tile).
__global__ void k_orb_lists(const int* __restrict__ gidx, int n_orb, int n_tiles, int mode,
                            int* __restrict__ cnt, const int* __restrict__ ptr,
                            int* __restrict__ list, int* __restrict__ slot) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_orb) return;
  int c = 0;
  int pos = mode ? ptr[o] : 0;
  for (int T = 0; T < n_tiles; ++T) {
    const int g = gidx[(size_t)o * n_tiles + T];
    if (g < 0) continue;
    ++c;
    if (mode) {
      list[pos] = T;
      slot[pos] = g;
      ++pos;
    }
  }
  if (!mode) cnt[o] = c;
}

__global__ void k_scan_small(const int* __restrict__ in, int n, int* __restrict__ out,
                             int* __restrict__ tot) {
  __shared__ long long part[1024];
  const int T = blockDim.x, chunk = (n + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(n, b + chunk);
  long long s = 0;
  for (int x = b; x < e; ++x) s += in[x];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < T; ++t) {
      long long v = part[t];
      part[t] = acc;
      acc += v;
    }
    *tot = (int)acc;
  }
  __syncthreads();
  long long pos = part[threadIdx.x];
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

__device__ __forceinline__ long long tile_point(const TileGeom& G, int T, int r) {
  const int txi = T % G.ntx, tyi = (T / G.ntx) % G.nty, tzi = T / (G.ntx * G.nty);
  const int x = txi * TX + (r % TX), y = tyi * TY + (r / TX) % TY, z = tzi * TZ + r / (TX * TY);
  if (x >= G.nx || y >= G.ny || z >= G.nz) return -1;
  return ((long long)z * G.ny + y) * G.nx + x;
}

// partial[(tptr[T] + s) * m + a] = sum_{r in T} A[a][r] W[list[s]][r].
// CTA per (tile, chunk of 64 rows of A); thread = (row a, quarter q) and
// accumulates the W rows q, q+4, q+8, ... of the tile's list (no padding:
// the quarter is uniform across a warp); W rows in blocks of 32, points
// staged 32 at a time in shared memory.
#define GA 64
#define GJ 32
#define GP 32
__global__ void __launch_bounds__(256)
    k_gram_partial(const double* __restrict__ A, int m, const double* __restrict__ W,
                   TileGeom G, size_t ng, const int* __restrict__ tptr,
                   const int* __restrict__ tlist, double* __restrict__ partial) {
  const int T = blockIdx.x;
  const int a0 = blockIdx.y * GA;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (nJ == 0) return;
  __shared__ double As[GA][GP + 1];
  __shared__ double Ws[GJ][GP + 1];
  __shared__ long long addr[TP];
  __shared__ int wrow[GJ];
  for (int r = threadIdx.x; r < TP; r += blockDim.x) addr[r] = tile_point(G, T, r);
  const int al = threadIdx.x % GA, qq = threadIdx.x / GA;
  for (int jb = 0; jb < nJ; jb += GJ) {
    const int nj = min(GJ, nJ - jb);
    double acc[GJ / 4];
#pragma unroll
    for (int u = 0; u < GJ / 4; ++u) acc[u] = 0.0;
    __syncthreads();
    if (threadIdx.x < nj) wrow[threadIdx.x] = tlist[j0 + jb + threadIdx.x];
    for (int pc = 0; pc < TP; pc += GP) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < GA * GP; idx += blockDim.x) {
        const int a = idx / GP, pt = idx % GP;
        const long long g = addr[pc + pt];
        As[a][pt] = (a0 + a < m && g >= 0) ? A[(size_t)(a0 + a) * ng + g] : 0.0;
      }
      for (int idx = threadIdx.x; idx < nj * GP; idx += blockDim.x) {
        const int jl = idx / GP, pt = idx % GP;
        const long long g = addr[pc + pt];
        Ws[jl][pt] = g >= 0 ? W[(size_t)wrow[jl] * ng + g] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int pt = 0; pt < GP; ++pt) {
        const double av = As[al][pt];
#pragma unroll
        for (int u = 0; u < GJ / 4; ++u)
          if (qq + 4 * u < nj) acc[u] = fma(av, Ws[qq + 4 * u][pt], acc[u]);
      }
    }
    if (a0 + al < m) {
#pragma unroll
      for (int u = 0; u < GJ / 4; ++u) {
        const int jl = qq + 4 * u;
        if (jl < nj) partial[(size_t)(j0 + jb + jl) * m + a0 + al] = acc[u];
      }
    }
  }
}

// out[a * sa + o * so] = scale * sum over the tiles of o (ascending) of
// partial[slot][a].
__global__ void k_gram_reduce(const double* __restrict__ partial, int m, int n_orb,
                              const int* __restrict__ optr, const int* __restrict__ oslot,
                              double scale, double* __restrict__ out, int sa, int so) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * n_orb) return;
  const int a = (int)(t % m), o = (int)(t / m);
  double s = 0.0;
  for (int k = optr[o]; k < optr[o + 1]; ++k) s += partial[(size_t)oslot[k] * m + a];
  out[(size_t)a * sa + (size_t)o * so] = scale * s;
}

// -Mbar = L L^T by a blocked right-looking Cholesky over several kernels
// (block 32): k_chol_init forms A = -(M + M^T)/2; per block column,
// k_chol_panel factors the 32 x 32 diagonal block in shared memory and
// solves the rows below it; k_chol_update subtracts the panel's
// contribution from the trailing lower triangle, one CTA per 32 x 32 block.
// A non-positive pivot sets SEA_FLAG_NOT_PD and the later kernels return.
#define CB 32
__global__ void k_chol_init(const double* __restrict__ M, int n, double* __restrict__ A) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int i = (int)(q / n), j = (int)(q % n);
  A[q] = (j <= i) ? -0.5 * (M[(size_t)i * n + j] + M[(size_t)j * n + i]) : 0.0;
}

__global__ void __launch_bounds__(256)
    k_chol_panel(double* __restrict__ A, int n, int kb, unsigned* __restrict__ status) {
  if (*status & SEA_FLAG_NOT_PD) return;
  __shared__ double D[CB][CB + 1];
  __shared__ int bad;
  const int nb = min(CB, n - kb);
  if (threadIdx.x == 0) bad = 0;
  for (int q = threadIdx.x; q < CB * CB; q += blockDim.x) {
    const int i = q / CB, j = q % CB;
    D[i][j] = (i < nb && j < nb) ? A[(size_t)(kb + i) * n + kb + j] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // one warp factors the diagonal block
    const int lane = threadIdx.x;
    for (int k = 0; k < nb; ++k) {
      double d = D[k][k];
      if (!(d > 0.0)) {
        if (lane == 0) bad = 1;
        break;
      }
      d = sqrt(d);
      __syncwarp();
      if (lane == 0) D[k][k] = d;
      if (lane > k && lane < nb) D[lane][k] /= d;
      __syncwarp();
      for (int j = k + 1; j < nb; ++j)
        if (lane >= j && lane < nb) D[lane][j] = fma(-D[lane][k], D[j][k], D[lane][j]);
      __syncwarp();
    }
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicOr(status, SEA_FLAG_NOT_PD);
    return;
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int i = q / nb, j = q % nb;
    if (j <= i) A[(size_t)(kb + i) * n + kb + j] = D[i][j];
  }
  // rows below: x L_kk^T = a  (forward substitution per row)
  for (int i = kb + nb + threadIdx.x; i < n; i += blockDim.x) {
    double x[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) x[j] = j < nb ? A[(size_t)i * n + kb + j] : 0.0;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      if (j < nb) {
        double v = x[j];
        for (int l = 0; l < j; ++l) v = fma(-x[l], D[j][l], v);
        x[j] = v / D[j][j];
      }
    }
#pragma unroll
    for (int j = 0; j < CB; ++j)
      if (j < nb) A[(size_t)i * n + kb + j] = x[j];
  }
}

__global__ void __launch_bounds__(256)
    k_chol_update(double* __restrict__ A, int n, int kb, const unsigned* __restrict__ status) {
  if (*status & SEA_FLAG_NOT_PD) return;
  // lower-triangular block (bi, bj), bj <= bi, of the trailing matrix
  const int t0 = kb + CB;
  const int nbt = (n - t0 + CB - 1) / CB;
  int bi = 0, rem = blockIdx.x;
  while (rem > bi) {
    rem -= bi + 1;
    ++bi;
  }
  const int bj = rem;
  if (bi >= nbt) return;
  __shared__ double Li[CB][CB + 1], Lj[CB][CB + 1];
  const int i0 = t0 + bi * CB, j0 = t0 + bj * CB;
  for (int q = threadIdx.x; q < CB * CB; q += blockDim.x) {
    const int r = q / CB, k = q % CB;
    Li[r][k] = (i0 + r < n) ? A[(size_t)(i0 + r) * n + kb + k] : 0.0;
    Lj[r][k] = (j0 + r < n) ? A[(size_t)(j0 + r) * n + kb + k] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < CB * CB; q += blockDim.x) {
    const int r = q / CB, cidx = q % CB;
    const int i = i0 + r, j = j0 + cidx;
    if (i >= n || j >= n || j > i) continue;
    double s = A[(size_t)i * n + j];
#pragma unroll 8
    for (int k = 0; k < CB; ++k) s = fma(-Li[r][k], Lj[cidx][k], s);
    A[(size_t)i * n + j] = s;
  }
}

// Column k of L^-1 by forward substitution, CTA per column.
__global__ void k_trinv(const double* __restrict__ L, int n, double* __restrict__ Linv) {
  extern __shared__ double xs[];
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (i == k) ? 1.0 : 0.0;
  __syncthreads();
  for (int l = k; l < n; ++l) {
    if (threadIdx.x == 0) xs[l] /= L[(size_t)l * n + l];
    __syncthreads();
    const double xl = xs[l];
    for (int i = l + 1 + threadIdx.x; i < n; i += blockDim.x) xs[i] = fma(-L[(size_t)i * n + l], xl, xs[i]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Linv[(size_t)i * n + k] = (i >= k) ? xs[i] : 0.0;
}

// C[n1][n2] = op(A) B, op(A)(i, k) = A[k][i] if transA else A[i][k]; A is
// n1 x n1 (square), B is [n1][n2].  16 x 16 shared-memory tiles.
__global__ void k_small_gemm(const double* __restrict__ A, int transA, const double* __restrict__ B,
                             int n1, int n2, double* __restrict__ C) {
  __shared__ double As[16][17], Bs[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < n1; k0 += 16) {
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

// out[v][r] = sign * sum_{j in tile list} W[j][r] H(j, v), H(j, v) =
// H[j * hj + v * hv], for every point r of the tile and v in a chunk of 32:
// thread = (point, half of the chunk), 16 accumulators.
#define EV 32
__global__ void __launch_bounds__(256)
    k_tile_expand(const double* __restrict__ W, TileGeom G, size_t ng,
                  const int* __restrict__ tptr, const int* __restrict__ tlist,
                  const double* __restrict__ H, long long hj, long long hv, int m, double sign,
                  double* __restrict__ out) {
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
  for (int jl = 0; jl < nJ; ++jl) {
    const double w = g >= 0 ? W[(size_t)tlist[j0 + jl] * ng + g] : 0.0;
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

static TileGeom tile_geom(const sea_ctx* c) {
  TileGeom G;
  G.nx = c->N[0];
  G.ny = c->N[1];
  G.nz = c->N[2];
  G.ntx = (G.nx + TX - 1) / TX;
  G.nty = (G.ny + TY - 1) / TY;
  G.ntz = (G.nz + TZ - 1) / TZ;
  return G;
}

// Tile lists of W's support, M, Cholesky and L^-1.  Needs the incidence
// count on the host to size the partial sums: one stream sync.
cudaError_t launch_ace_build(sea_ctx* c) {
  const int n = c->n_orb;
  const TileGeom G = tile_geom(c);
  const int nt = G.ntx * G.nty * G.ntz;
  c->n_tiles = nt;
  const long long ninc = (long long)n * nt;
  if (!sea_ensure(c, c->tmask, ninc * sizeof(int) * 2) ||
      !sea_ensure(c, c->tptr_t, (size_t)(nt + 1) * sizeof(int) * 2) ||
      !sea_ensure(c, c->tptr_o, (size_t)(n + 1) * sizeof(int) * 2) ||
      !sea_ensure(c, c->Mbuf, (size_t)n * n * sizeof(double)) ||
      !sea_ensure(c, c->Lbuf, (size_t)n * n * sizeof(double)) ||
      !sea_ensure(c, c->Linv, (size_t)n * n * sizeof(double)))
    return cudaErrorMemoryAllocation;
  int* inc = (int*)c->tmask.p;
  int* gidx = inc + ninc;
  int* tcnt = (int*)c->tptr_t.p;
  int* tptr = tcnt + (nt + 1);
  int* ocnt = (int*)c->tptr_o.p;
  int* optr = ocnt + (n + 1);
  int* counts = (int*)c->counts.p;
  k_tile_incidence<<<(unsigned)((ninc + 255) / 256), 256, 0, c->stream>>>(
      (const Entry*)c->ewin.p, (const int*)c->eptr.p, n, G, nt, inc);
  k_tile_lists<<<(nt + 127) / 128, 128, 0, c->stream>>>(inc, n, nt, 0, tcnt, nullptr, nullptr,
                                                        nullptr);
  k_scan_small<<<1, 1024, 0, c->stream>>>(tcnt, nt, tptr, counts + 10);
  k_max_int<<<1, 1024, 0, c->stream>>>(tcnt, nt, counts + 12);
  int hc[3] = {0, 0, 0};
  cudaMemcpyAsync(hc, counts + 10, sizeof(hc), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t err = cudaStreamSynchronize(c->stream);
  if (err != cudaSuccess) return err;
  const int hinc = hc[0];
  c->tile_inc = hinc;
  c->max_tile_list = hc[2];
  {
    const size_t smem = (size_t)c->max_tile_list * EV * sizeof(double);
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(k_tile_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
      if (err != cudaSuccess) return err;
    }
  }
  if (!sea_ensure(c, c->tlist_t, (size_t)max(hinc, 1) * sizeof(int)) ||
      !sea_ensure(c, c->tlist_o, (size_t)max(hinc, 1) * sizeof(int) * 2) ||
      !sea_ensure(c, c->partial, (size_t)max(hinc, 1) * n * sizeof(double)))
    return cudaErrorMemoryAllocation;
  int* tlist = (int*)c->tlist_t.p;
  int* olist = (int*)c->tlist_o.p;
  int* oslot = olist + max(hinc, 1);
  k_tile_lists<<<(nt + 127) / 128, 128, 0, c->stream>>>(inc, n, nt, 1, nullptr, tptr, tlist, gidx);
  k_orb_lists<<<(n + 127) / 128, 128, 0, c->stream>>>(gidx, n, nt, 0, ocnt, nullptr, nullptr,
                                                      nullptr);
  k_scan_small<<<1, 1024, 0, c->stream>>>(ocnt, n, optr, counts + 11);
  k_orb_lists<<<(n + 127) / 128, 128, 0, c->stream>>>(gidx, n, nt, 1, nullptr, optr, olist, oslot);
  // M = Phi^T W dV
  k_gram_partial<<<dim3(nt, (n + GA - 1) / GA), 256, 0, c->stream>>>(
      (const double*)c->phi.p, n, (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist,
      (double*)c->partial.p);
  k_gram_reduce<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, c->stream>>>(
      (const double*)c->partial.p, n, n, optr, oslot, c->dV, (double*)c->Mbuf.p, n, 1);
  k_chol_init<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, c->stream>>>(
      (const double*)c->Mbuf.p, n, (double*)c->Lbuf.p);
  int nchol = 1;
  for (int kb = 0; kb < n; kb += CB) {
    k_chol_panel<<<1, 256, 0, c->stream>>>((double*)c->Lbuf.p, n, kb, (unsigned*)c->status.p);
    const int nbt = (n - kb - CB + CB - 1) / CB;
    if (nbt > 0)
      k_chol_update<<<nbt * (nbt + 1) / 2, 256, 0, c->stream>>>((double*)c->Lbuf.p, n, kb,
                                                                 (const unsigned*)c->status.p);
    nchol += 1 + (nbt > 0);
  }
  k_trinv<<<n, 256, n * sizeof(double), c->stream>>>((const double*)c->Lbuf.p, n,
                                                     (double*)c->Linv.p);
  c->launches += 11 + nchol;
  return cudaGetLastError();
}

cudaError_t launch_ace_apply(sea_ctx* c, const double* psi, int nv, double* out) {
  const int n = c->n_orb;
  const TileGeom G = tile_geom(c);
  const int nt = c->n_tiles;
  const int hinc = c->tile_inc;
  if (!sea_ensure(c, c->partial, (size_t)max(hinc, 1) * max(n, nv) * sizeof(double)) ||
      !sea_ensure(c, c->Gbuf, (size_t)n * nv * sizeof(double)) ||
      !sea_ensure(c, c->Hbuf, (size_t)n * nv * sizeof(double)) ||
      !sea_ensure(c, c->Hbuf2, (size_t)n * nv * sizeof(double)))
    return cudaErrorMemoryAllocation;
  const int* tptr = (const int*)c->tptr_t.p + (nt + 1);
  const int* tlist = (const int*)c->tlist_t.p;
  const int* optr = (const int*)c->tptr_o.p + (n + 1);
  const int* olist = (const int*)c->tlist_o.p;
  const int* oslot = olist + max(hinc, 1);
  // G[o][v] = <W_o|psi_v> dV
  k_gram_partial<<<dim3(nt, (nv + GA - 1) / GA), 256, 0, c->stream>>>(
      psi, nv, (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist, (double*)c->partial.p);
  k_gram_reduce<<<(unsigned)(((long long)n * nv + 255) / 256), 256, 0, c->stream>>>(
      (const double*)c->partial.p, nv, n, optr, oslot, c->dV, (double*)c->Gbuf.p, 1, nv);
  // H = L^-T (L^-1 G)
  dim3 gb((nv + 15) / 16, (n + 15) / 16), tb(16, 16);
  k_small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 0, (const double*)c->Gbuf.p, n,
                                         nv, (double*)c->Hbuf2.p);
  k_small_gemm<<<gb, tb, 0, c->stream>>>((const double*)c->Linv.p, 1, (const double*)c->Hbuf2.p, n,
                                         nv, (double*)c->Hbuf.p);
  // out[v] = -sum_j W_j H[j][v]
  const size_t smem = (size_t)c->max_tile_list * EV * sizeof(double);
  k_tile_expand<<<dim3(nt, (nv + EV - 1) / EV), 256, smem, c->stream>>>(
      (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist, (const double*)c->Hbuf.p, nv, 1, nv,
      -1.0, out);
  c->launches += 5;
  return cudaGetLastError();
}

cudaError_t launch_ace_vectors(sea_ctx* c, double* xi) {
  const int n = c->n_orb;
  const TileGeom G = tile_geom(c);
  const int nt = c->n_tiles;
  const int* tptr = (const int*)c->tptr_t.p + (nt + 1);
  const int* tlist = (const int*)c->tlist_t.p;
  const size_t smem = (size_t)c->max_tile_list * EV * sizeof(double);
  // Xi[k][r] = sum_j W[j][r] (L^-1)[k][j]:  H(j, k) = Linv[k * n + j]
  k_tile_expand<<<dim3(nt, (n + EV - 1) / EV), 256, smem, c->stream>>>(
      (const double*)c->vxx_dev.p, G, c->ng, tptr, tlist, (const double*)c->Linv.p, 1, n, n, 1.0,
      xi);
  c->launches += 1;
  return cudaGetLastError();
}

}  // namespace sea
