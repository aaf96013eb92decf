// plan.cu -- domain truncation (Eq. oii) and pair selection (Eq. sij).
//
// Both steps end in integer decisions taken on FP64 sums.  Every sum here
// is either exact or has a fixed order and a fixed rounding (explicit fma,
// or __dmul_rn / __dadd_rn where no fusion is wanted), so the decisions do
// not depend on the launch shape and match the oracle bit for bit:
//   marginals m_a(x) = fl(fl(2^-64 sum F(phi)) dV) with the exact integer
//   sums of F(v) = min(floor(v^2 2^64), 2^96) over each plane normal to
//   axis a; the box of each axis is the shortest cyclic interval whose
//   outside mass T - inside <= eps/3, inside summed from the interval
//   start upward, T the ascending total (ties: lowest start); S_|ij| sums
//   |phi_i phi_j| over each (z, y) row of Omega_ij in x order, then the
//   rows in (z, y) order, then multiplies by dV.
#include "sea_internal.cuh"

namespace sea {

// F(v) = min(floor(v^2 2^64), 2^96), exactly, as two 48-bit limbs
// (F = lo + hi 2^48).  |v| = m 2^(eb - 1075) with the 53-bit significand m
// and biased exponent eb, so F = floor(m^2 2^(2 eb - 2086)); subnormals and
// zeros give 0, |v| >= 2^16 (eb >= 1039) saturates.  Integer operations only.
__device__ __forceinline__ void sq_fixed(double v, unsigned long long& lo, unsigned long long& hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int r = 2086 - 2 * eb;  // right shift of m^2
  if (eb == 0 || r >= 106) {
    lo = hi = 0;
    return;
  }
  if (eb >= 1039) {
    lo = 0;
    hi = 1ULL << 48;
    return;
  }
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const unsigned long long ml = m & 0xFFFFFFFFULL, mh = m >> 32;  // mh < 2^21
  // m^2 = P1 2^64 + P0 (128-bit)
  const unsigned long long a0 = ml * ml, a1 = mh * ml, a2 = mh * mh;
  unsigned long long P0 = a0 + (a1 << 33);
  unsigned long long P1 = a2 + (a1 >> 31) + (P0 < a0 ? 1ULL : 0ULL);
  // F = (P1 2^64 + P0) >> r, r in [10, 106)
  unsigned long long F0, F1;
  if (r < 64) {
    F0 = (P0 >> r) | (P1 << (64 - r));
    F1 = P1 >> r;
  } else {
    F0 = P1 >> (r - 64);
    F1 = 0;
  }
  lo = F0 & 0xFFFFFFFFFFFFULL;
  hi = (F0 >> 48) | (F1 << 16);
}

// One CTA of four warps per (z-plane, orbital): row sums and column sums of
// F(phi) over the plane, as 48-bit limb sums (exact: a row or column has at
// most 1024 points).  The plane is staged through shared memory as F values
// in chunks of whole rows (coalesced loads, one chunk ahead in registers;
// row pitch nx + 1 so that lanes reading different rows hit distinct
// banks).  Warp w sums quarter w of every row of the chunk (lane per row),
// the quarters are then added; thread per column carries the column sums
// over the chunks in shared memory.  All sums are exact, so the split is
// free.
#define RC_ROWS 32
#define RC_SMEM_ELEMS 3200
#define RC_PER_THREAD (RC_SMEM_ELEMS / 128)  // tile elements per thread (128 threads)
__host__ __device__ __forceinline__ int rc_rows(int nx) {
  return min(RC_ROWS, max(1, (RC_SMEM_ELEMS - nx) / (nx + 1)));
}
__host__ __forceinline__ size_t rc_smem_bytes(int nx) {
  return ((size_t)rc_rows(nx) * (nx + 1) + nx) * sizeof(ulonglong2);
}

__global__ void __launch_bounds__(128)
    k_row_col_sums(const double* __restrict__ phi, int nx, int ny, int nz,
                   ulonglong2* __restrict__ R, ulonglong2* __restrict__ C) {
  extern __shared__ ulonglong2 rc_sm[];  // [rows][nx + 1] F tile, then [nx] column sums
  __shared__ ulonglong2 rpart[4 * RC_ROWS];  // row partial sums, one per warp
  const int pitch = nx + 1;
  const int rows = rc_rows(nx);
  ulonglong2* tile = rc_sm;
  ulonglong2* col = rc_sm + rows * pitch;
  const int z = blockIdx.x, i = blockIdx.y;
  const double* plane = phi + ((size_t)i * nz + z) * (size_t)ny * nx;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dqr = 128 / nx, dqx = 128 - dqr * nx;  // the step of 128 elements in rows and columns
  for (int x = threadIdx.x; x < nx; x += blockDim.x) col[x] = make_ulonglong2(0, 0);
  // a chunk's values are loaded into registers one chunk ahead, so the loads
  // of chunk k + 1 are in flight while chunk k is summed
  double v[RC_PER_THREAD];
  auto load_chunk = [&](int y0) {
    const int nq = min(rows, ny - y0) * nx;
    const double* src = plane + (size_t)y0 * nx;
#pragma unroll
    for (int u = 0; u < RC_PER_THREAD; ++u) {
      const int q = threadIdx.x + u * 128;
      v[u] = q < nq ? src[q] : 0.0;
    }
  };
  load_chunk(0);
  for (int y0 = 0; y0 < ny; y0 += rows) {
    const int nr = min(rows, ny - y0);
    __syncthreads();  // the previous chunk's tile is no longer read
    const int nq = nr * nx;
    // (row, column) of element q = tid + 128 u, advanced without divisions
    int r = threadIdx.x / nx, x = threadIdx.x - r * nx;
#pragma unroll
    for (int u = 0; u < RC_PER_THREAD; ++u) {
      if (threadIdx.x + u * 128 < nq) {
        unsigned long long lo, hi;
        sq_fixed(v[u], lo, hi);
        tile[r * pitch + x] = make_ulonglong2(lo, hi);
      }
      x += dqx;
      r += dqr;
      if (x >= nx) {
        x -= nx;
        ++r;
      }
    }
    __syncthreads();
    if (y0 + rows < ny) load_chunk(y0 + rows);
    // row sums: warp w adds quarter w of every row (lane = row); the four
    // partial sums are exact, so their combination below is too
    const int qx = (nx + 3) / 4, xa = w * qx, xb = min(nx, xa + qx);
    if (lane < nr) {
      unsigned long long slo = 0, shi = 0;
      for (int x = xa; x < xb; ++x) {
        const ulonglong2 f = tile[lane * pitch + x];
        slo += f.x;
        shi += f.y;
      }
      rpart[w * 32 + lane] = make_ulonglong2(slo, shi);
    }
    // column sums: thread per column, carried over the chunks
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      ulonglong2 c = col[x];
      for (int r = 0; r < nr; ++r) {
        const ulonglong2 f = tile[r * pitch + x];
        c.x += f.x;
        c.y += f.y;
      }
      col[x] = c;
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      ulonglong2 t = rpart[threadIdx.x];
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        t.x += rpart[u * 32 + threadIdx.x].x;
        t.y += rpart[u * 32 + threadIdx.x].y;
      }
      R[((size_t)i * nz + z) * ny + y0 + threadIdx.x] = t;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nx; x += blockDim.x) C[((size_t)i * nz + z) * nx + x] = col[x];
}

// The same sums without a shared-memory tile, for rows of at most 32 KX
// points: warp w takes the rows y = w, w + 4, ... (two at a time), lane l
// the points x = l + 32 k; a row's sum is a warp butterfly, a column's
// partial sums stay in the lane's registers until one exchange between the
// four warps at the end of the plane.  All sums are exact, so the order is
// free.
template <int KX>
__global__ void __launch_bounds__(128)
    k_row_col_sums_reg(const double* __restrict__ phi, int nx, int ny, int nz,
                       ulonglong2* __restrict__ R, ulonglong2* __restrict__ C) {
  __shared__ ulonglong2 cpart[4][32 * KX];  // per warp: column partial sums
  const int z = blockIdx.x, i = blockIdx.y;
  const double* plane = phi + ((size_t)i * nz + z) * (size_t)ny * nx;
  ulonglong2* Rp = R + ((size_t)i * nz + z) * ny;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long clo[KX], chi[KX];
#pragma unroll
  for (int k = 0; k < KX; ++k) clo[k] = chi[k] = 0;
  for (int y0 = w; y0 < ny; y0 += 8) {
    double v[2][KX];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int y = y0 + 4 * t;
      const double* row = plane + (size_t)y * nx;
#pragma unroll
      for (int k = 0; k < KX; ++k) {
        const int x = lane + 32 * k;
        v[t][k] = (y < ny && x < nx) ? row[x] : 0.0;
      }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      unsigned long long rlo = 0, rhi = 0;
#pragma unroll
      for (int k = 0; k < KX; ++k) {
        unsigned long long lo, hi;
        sq_fixed(v[t][k], lo, hi);
        clo[k] += lo;
        chi[k] += hi;
        rlo += lo;
        rhi += hi;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        rlo += __shfl_xor_sync(0xffffffffu, rlo, o);
        rhi += __shfl_xor_sync(0xffffffffu, rhi, o);
      }
      const int y = y0 + 4 * t;
      if (lane == 0 && y < ny) Rp[y] = make_ulonglong2(rlo, rhi);
    }
  }
#pragma unroll
  for (int k = 0; k < KX; ++k) cpart[w][32 * k + lane] = make_ulonglong2(clo[k], chi[k]);
  __syncthreads();
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    ulonglong2 c = cpart[0][x];
#pragma unroll
    for (int u = 1; u < 4; ++u) {
      c.x += cpart[u][x].x;
      c.y += cpart[u][x].y;
    }
    C[((size_t)i * nz + z) * nx + x] = c;
  }
}

// 128-bit unsigned (hi, lo) += limb pair (a + b 2^48).
__device__ __forceinline__ void add_limbs(unsigned long long& hi, unsigned long long& lo,
                                          ulonglong2 v) {
  const unsigned long long b_lo = v.y << 48, b_hi = v.y >> 16;
  unsigned long long t = lo + v.x;
  hi += (t < lo ? 1ULL : 0ULL);
  const unsigned long long t2 = t + b_lo;
  hi += (t2 < t ? 1ULL : 0ULL) + b_hi;
  lo = t2;
}

// (hi 2^64 + lo) 2^e2 rounded to the nearest FP64 value (ties to even);
// integer operations only.  0 for a zero input.
__device__ __forceinline__ double scaled_u128(unsigned long long hi, unsigned long long lo, int e2) {
  if (hi == 0 && lo == 0) return 0.0;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  unsigned long long H, L;
  if (lz >= 64) {
    H = lo << (lz - 64);
    L = 0;
  } else if (lz > 0) {
    H = (hi << lz) | (lo >> (64 - lz));
    L = lo << lz;
  } else {
    H = hi;
    L = lo;
  }
  unsigned long long mnt = H >> 11;
  const unsigned rem = (unsigned)(H & 0x7FF);
  if (rem > 0x400u || (rem == 0x400u && (L != 0 || (mnt & 1ULL)))) ++mnt;
  int ex = 127 - lz + e2 + 1023;
  if (mnt >> 53) {
    mnt >>= 1;
    ++ex;
  }
  if (ex <= 0) return 0.0;
  return __longlong_as_double((long long)(((unsigned long long)ex << 52) | (mnt & 0xFFFFFFFFFFFFFULL)));
}

// The three marginals of |phi|^2 dV, m = fl(fl(2^-64 S) dV) with S the exact
// sum of the plane's F values (integer sums: any grouping gives the same S).
// A CTA per (orbital, axis).  z (sum over y of the row sums R[i][z][y],
// contiguous): a warp per z, lanes over y, a warp reduction.  y and x (sums
// over z of R[i][z][y] and C[i][z][x]): a thread per (coordinate, part of
// the z range), loads coalesced over the coordinate, the parts added in
// shared memory.  marg layout: [n][3][Nmax].
__device__ __forceinline__ void add_u128(unsigned long long& hi, unsigned long long& lo,
                                         unsigned long long h2, unsigned long long l2) {
  const unsigned long long t = lo + l2;
  hi += h2 + (t < lo ? 1ULL : 0ULL);
  lo = t;
}
constexpr int MG_THREADS = 256;
__global__ void __launch_bounds__(MG_THREADS)
    k_marginals(const ulonglong2* __restrict__ R, const ulonglong2* __restrict__ C, int n, int nx,
                int ny, int nz, int Nmax, double dV, double* __restrict__ marg) {
  extern __shared__ unsigned long long mg_part[];  // [parts][2 Nmax]
  const int axis = blockIdx.x % 3, i = blockIdx.x / 3;
  double* out = marg + ((size_t)i * 3 + axis) * Nmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (axis == 2) {
    for (int z = warp; z < nz; z += MG_THREADS / 32) {
      const ulonglong2* r = R + ((size_t)i * nz + z) * ny;
      unsigned long long hi = 0, lo = 0;
      for (int y = lane; y < ny; y += 32) add_limbs(hi, lo, r[y]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        add_u128(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
      if (lane == 0) out[z] = __dmul_rn(scaled_u128(hi, lo, -64), dV);
    }
    return;
  }
  const int m = axis == 1 ? ny : nx;  // coordinates of this marginal
  const ulonglong2* src = axis == 1 ? R : C;
  const int parts = max(1, MG_THREADS / m);
  for (int c = threadIdx.x; c < m * parts; c += MG_THREADS) {
    const int coord = c % m, p = c / m;
    const int z0 = (int)((long long)nz * p / parts), z1 = (int)((long long)nz * (p + 1) / parts);
    unsigned long long hi = 0, lo = 0;
    const ulonglong2* col = src + ((size_t)i * nz) * m + coord;
    int z = z0;
    for (; z + 4 <= z1; z += 4) {
      const ulonglong2 v0 = col[(size_t)z * m], v1 = col[(size_t)(z + 1) * m];
      const ulonglong2 v2 = col[(size_t)(z + 2) * m], v3 = col[(size_t)(z + 3) * m];
      add_limbs(hi, lo, v0);
      add_limbs(hi, lo, v1);
      add_limbs(hi, lo, v2);
      add_limbs(hi, lo, v3);
    }
    for (; z < z1; ++z) add_limbs(hi, lo, col[(size_t)z * m]);
    mg_part[2 * ((size_t)p * Nmax + coord)] = hi;
    mg_part[2 * ((size_t)p * Nmax + coord) + 1] = lo;
  }
  __syncthreads();
  for (int coord = threadIdx.x; coord < m; coord += MG_THREADS) {
    unsigned long long hi = 0, lo = 0;
    for (int p = 0; p < parts; ++p)
      add_u128(hi, lo, mg_part[2 * ((size_t)p * Nmax + coord)], mg_part[2 * ((size_t)p * Nmax + coord) + 1]);
    out[coord] = __dmul_rn(scaled_u128(hi, lo, -64), dV);
  }
}

// One CTA per (orbital, axis): shortest cyclic interval with outside mass
// <= tail.  Thread per start s finds its shortest length (the condition is
// monotone in the length: inside only grows); then the lexicographic
// minimum of (length, start).  A start stops once its length reaches the
// shortest one found so far by any start (it can no longer win), which
// leaves every decision and sum as they were.  No interval at all
// (possible only for tail = 0 under rounding): the whole axis from 0.
__global__ void k_box_fit(const double* __restrict__ marg, int nx, int ny, int nz, int Nmax,
                          double tail, int* __restrict__ box) {
  extern __shared__ double sm[];
  const int axis = blockIdx.x % 3, i = blockIdx.x / 3;
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const double* m = marg + ((size_t)i * 3 + axis) * Nmax;
  for (int x = threadIdx.x; x < n; x += blockDim.x) sm[x] = m[x];
  __shared__ double sT;
  __shared__ long long sbest[32];
  __shared__ int sbestL;  // shortest length found so far (only decreases)
  __syncthreads();
  if (threadIdx.x == 0) {
    double T = 0.0;
    for (int x = 0; x < n; ++x) T = __dadd_rn(T, sm[x]);
    sT = T;
    sbestL = n;
  }
  __syncthreads();
  const double T = sT;
  const volatile int* vbest = &sbestL;
  long long best = 0x7fffffffffffffffLL;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    double inside = 0.0;
    int L = 0, found = 0;
    while (L < n) {
      if (L >= *vbest) break;  // its length would exceed the shortest found
      int x = s + L;
      if (x >= n) x -= n;
      inside = __dadd_rn(inside, sm[x]);
      ++L;
      if (__dsub_rn(T, inside) <= tail) {
        found = 1;
        atomicMin(&sbestL, L);
        break;
      }
    }
    if (found) {
      long long key = (long long)L * 4096 + s;
      if (key < best) best = key;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long other = __shfl_xor_sync(0xffffffffu, best, o);
    if (other < best) best = other;
  }
  if ((threadIdx.x & 31) == 0) sbest[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long b = sbest[0];
    for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w)
      if (sbest[w] < b) b = sbest[w];
    int s0 = 0, L0 = n;
    if (b != 0x7fffffffffffffffLL) {
      L0 = (int)(b / 4096);
      s0 = (int)(b % 4096);
    }
    box[i * 6 + axis] = s0;
    box[i * 6 + 3 + axis] = L0;
  }
}

// Intersection of cyclic intervals (reading of the wrap-around case): j's
// interval shifted by k n, k in {-1, 0, 1}; keep the largest overlap (first
// k on ties); a full-axis interval leaves the other one as it is.
__device__ bool interval_meet(int s1, int L1, int s2, int L2, int n, int* lo, int* ext,
                              int* kk) {
  if (L1 >= n && L2 >= n) { *lo = s1; *ext = n; *kk = 0; return true; }
  if (L1 >= n) { *lo = s2; *ext = L2; *kk = 0; return true; }
  if (L2 >= n) { *lo = s1; *ext = L1; *kk = 0; return true; }
  int best = 0, bk = 0, blo = 0;
  for (int k = -1; k <= 1; ++k) {
    int a0 = max(s1, s2 + k * n);
    int a1 = min(s1 + L1, s2 + k * n + L2);
    if (a1 - a0 > best) { best = a1 - a0; bk = k; blo = a0; }
  }
  if (best <= 0) return false;
  *lo = blo; *ext = best; *kk = bk;
  return true;
}

// Candidate c enumerates i <= j row by row: c = i n - i(i-1)/2 + (j - i).
__device__ __forceinline__ void decode_pair(long long c, int n, int* pi, int* pj) {
  // row i starts at off(i) = i n - i(i-1)/2; find the last row with off <= c
  double b = 2.0 * n + 1.0;
  int i = (int)floor((b - sqrt(b * b - 8.0 * (double)c)) * 0.5);
  if (i < 0) i = 0;
  if (i > n - 1) i = n - 1;
  while (i > 0 && (long long)i * n - (long long)i * (i - 1) / 2 > c) --i;
  while (i + 1 < n && (long long)(i + 1) * n - (long long)(i + 1) * i / 2 <= c) ++i;
  *pi = i;
  *pj = i + (int)(c - ((long long)i * n - (long long)i * (i - 1) / 2));
}

// geom layout per candidate: lo[3], ext[3], k[3].
__global__ void k_proto_pairs(const int* __restrict__ box, int n, int nx, int ny, int nz,
                              long long ncand, int* __restrict__ flag, int* __restrict__ geom) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  int i, j;
  decode_pair(c, n, &i, &j);
  const int N[3] = {nx, ny, nz};
  int g[9];
  bool ok = true;
  for (int a = 0; a < 3 && ok; ++a)
    ok = interval_meet(box[i * 6 + a], box[i * 6 + 3 + a], box[j * 6 + a], box[j * 6 + 3 + a],
                       N[a], &g[a], &g[3 + a], &g[6 + a]);
  flag[c] = ok ? 1 : 0;
  if (ok)
    for (int q = 0; q < 9; ++q) geom[c * 9 + q] = g[q];
}

// Single-CTA stable compaction: out[k] = index of the k-th set flag;
// *count = number of set flags.  Each thread scans a contiguous chunk.
__global__ void k_compact(const int* __restrict__ flag, long long n_host,
                          const int* __restrict__ n_dev, int* __restrict__ out,
                          int* __restrict__ count) {
  __shared__ long long part[32];
  const long long n = n_dev ? (long long)*n_dev : n_host;
  const int T = blockDim.x;
  const long long chunk = (n + T - 1) / T;
  const long long b = chunk * threadIdx.x;
  const long long e = min(n, b + chunk);
  long long s = 0;
  for (long long x = b; x < e; ++x) s += flag[x] != 0;
  long long acc = 0;
  long long pos = block_exscan_ll(s, part, &acc);
  if (threadIdx.x == 0) *count = (int)acc;
  for (long long x = b; x < e; ++x)
    if (flag[x]) out[pos++] = (int)x;
}

// A CTA per proto-pair (CTA-stride loop over them): S_|ij| in the fixed row
// order, keep decision.
__global__ void k_screen(const double* __restrict__ phi, int n, int nx, int ny, int nz,
                         const int* __restrict__ proto_list, const int* __restrict__ nproto,
                         const int* __restrict__ geom, double dV, double delta,
                         int* __restrict__ keep, double* __restrict__ Sout) {
  const int np = *nproto;
  __shared__ double rows[1024];
  __shared__ double tot;
  for (int q = blockIdx.x; q < np; q += gridDim.x) {  // CTA-stride over the proto-pairs
    __syncthreads();  // rows and tot of the previous proto-pair are consumed
    const long long c = proto_list[q];
    int i, j;
    decode_pair(c, n, &i, &j);
    const int* g = geom + c * 9;
    const int ex = g[3], ey = g[4], ez = g[5];
    const size_t ng = (size_t)nx * ny * nz;
    const double* fi = phi + (size_t)i * ng;
    const double* fj = phi + (size_t)j * ng;
    if (threadIdx.x == 0) tot = 0.0;
    const int nrows = ey * ez;
    for (int r0 = 0; r0 < nrows; r0 += 1024) {
      __syncthreads();
      for (int r = r0 + threadIdx.x; r < min(nrows, r0 + 1024); r += blockDim.x) {
        const int y = r % ey, z = r / ey;
        const int gz = wrapi(g[2] + z, nz), gy = wrapi(g[1] + y, ny);
        const size_t base = ((size_t)gz * ny + gy) * nx;
        double row = 0.0;
        for (int x = 0; x < ex; ++x) {
          const int gx = wrapi(g[0] + x, nx);
          row = __dadd_rn(row, fabs(__dmul_rn(fi[base + gx], fj[base + gx])));
        }
        rows[r - r0] = row;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = tot;
        for (int r = r0; r < min(nrows, r0 + 1024); ++r) t = __dadd_rn(t, rows[r - r0]);
        tot = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double S = __dmul_rn(tot, dV);
      Sout[q] = S;
      keep[q] = (i == j || S >= delta) ? 1 : 0;
    }
  }
}

// Build the pair records in (i, j) order from the kept proto-pairs.
__global__ void k_fill_pairs(const int* __restrict__ kept, const int* __restrict__ npairs,
                             const int* __restrict__ proto_list, const int* __restrict__ geom,
                             const double* __restrict__ Sproto, int n, PairInfo* __restrict__ pinfo,
                             double* __restrict__ S, int* __restrict__ pn) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= *npairs) return;
  const int q = kept[p];
  const long long c = proto_list[q];
  int i, j;
  decode_pair(c, n, &i, &j);
  const int* g = geom + c * 9;
  PairInfo P;
  P.i = i;
  P.j = j;
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = g[a];
    P.ext[a] = g[3 + a];
    P.k[a] = g[6 + a];
  }
  P.n = P.ext[0] * P.ext[1] * P.ext[2];
  pinfo[p] = P;
  S[p] = Sproto[q];
  pn[p] = P.n;
}

// Single-CTA exclusive scan of P sizes into 64-bit offsets; total in *tot,
// and the largest pair box in the mixed CG's padded shared-memory layout
// (ex (ey + F)(ez + 2F) floats, F = SEA_FDP) in *maxpad.
__global__ void k_scan_sizes(const int* __restrict__ sz, const int* __restrict__ count,
                             const PairInfo* __restrict__ pinfo, long long* __restrict__ off,
                             long long* __restrict__ tot, int* __restrict__ maxpad) {
  __shared__ long long part[32];
  const int n = *count;
  const int T = blockDim.x;
  const int chunk = (n + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(n, b + chunk);
  long long s = 0;
  int pm = 0;
  for (int x = b; x < e; ++x) {
    s += sz[x];
    const PairInfo P = pinfo[x];
    pm = max(pm, P.ext[0] * (P.ext[1] + SEA_FDP) * (P.ext[2] + 2 * SEA_FDP));
  }
  long long acc = 0;
  long long pos = block_exscan_ll(s, part, &acc);
  const int m = (int)block_max_ll(pm, part);
  if (threadIdx.x == 0) {
    *tot = acc;
    *maxpad = m;
  }
  for (int x = b; x < e; ++x) {
    off[x] = pos;
    pos += sz[x];
  }
}

// Longest-first processing order for the CG queue: rank by (size desc,
// index asc).  The sizes pass through shared memory in chunks, read by all
// threads at once (broadcast).
__global__ void __launch_bounds__(256) k_lpt_order(const int* __restrict__ sz,
                                                   const int* __restrict__ count,
                                                   int* __restrict__ order) {
  __shared__ int s_sz[2048];
  const int n = *count;
  if ((int)(blockIdx.x * blockDim.x) >= n) return;  // uniform over the CTA
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int mine = p < n ? sz[p] : 0;
  int rank = 0;
  for (int q0 = 0; q0 < n; q0 += 2048) {
    const int m = min(2048, n - q0);
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += blockDim.x) s_sz[q] = sz[q0 + q];
    __syncthreads();
    for (int q = 0; q < m; ++q) {
      const int o = s_sz[q];
      rank += (o > mine) || (o == mine && q0 + q < p);
    }
  }
  if (p < n) order[rank] = p;
}

cudaError_t launch_plan_boxes(sea_ctx* c) {
  const int n = c->n_orb, nx = c->N[0], ny = c->N[1], nz = c->N[2];
  const int Nmax = max(nx, max(ny, nz));
  const dim3 rc_grid(nz, n);
  const double* phi = (const double*)c->phi.p;
  ulonglong2* Rs = (ulonglong2*)c->rowsum.p;
  ulonglong2* Cs = (ulonglong2*)c->colsum.p;
  if (nx <= 64)
    k_row_col_sums_reg<2><<<rc_grid, 128, 0, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  else if (nx <= 96)
    k_row_col_sums_reg<3><<<rc_grid, 128, 0, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  else if (nx <= 128)
    k_row_col_sums_reg<4><<<rc_grid, 128, 0, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  else if (nx <= 192)
    k_row_col_sums_reg<6><<<rc_grid, 128, 0, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  else if (nx <= 256)
    k_row_col_sums_reg<8><<<rc_grid, 128, 0, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  else {
    const size_t rc_smem = rc_smem_bytes(nx);
    cudaError_t e = cudaFuncSetAttribute(k_row_col_sums, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rc_smem);
    if (e != cudaSuccess) return e;
    k_row_col_sums<<<rc_grid, 128, rc_smem, c->stream>>>(phi, nx, ny, nz, Rs, Cs);
  }
  {
    const int mmin = std::max(1, std::min(nx, ny));
    const size_t mg_smem = (size_t)std::max(1, MG_THREADS / mmin) * Nmax * 2 * sizeof(unsigned long long);
    if (mg_smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_marginals, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)mg_smem);
      if (e != cudaSuccess) return e;
    }
    k_marginals<<<n * 3, MG_THREADS, mg_smem, c->stream>>>(
        (const ulonglong2*)c->rowsum.p, (const ulonglong2*)c->colsum.p, n, nx, ny, nz, Nmax,
        c->dV, (double*)c->marg.p);
  }
  k_box_fit<<<n * 3, 128, Nmax * sizeof(double), c->stream>>>(
      (const double*)c->marg.p, nx, ny, nz, Nmax, c->prm.eps / 3.0, (int*)c->box.p);
  c->launches += 3;
  return cudaGetLastError();
}

// Candidates, proto-pair compaction, screening, kept compaction, pair
// records, unknown offsets and the CG order, all with device-side counts:
// counts[0] = proto pairs, counts[1] = pairs, *(long long*)(counts + 4) =
// total unknowns, counts[10] = largest padded pair box.  Grids are sized for the worst case (every candidate).
cudaError_t launch_plan_pairs(sea_ctx* c) {
  const int n = c->n_orb;
  const long long ncand = (long long)n * (n + 1) / 2;
  const unsigned gc = (unsigned)((ncand + 255) / 256);
  int* counts = (int*)c->counts.p;
  k_proto_pairs<<<gc, 256, 0, c->stream>>>((const int*)c->box.p, n, c->N[0], c->N[1], c->N[2],
                                           ncand, (int*)c->cand_flag.p, (int*)c->cand_geom.p);
  k_compact<<<1, 1024, 0, c->stream>>>((const int*)c->cand_flag.p, ncand, nullptr,
                                       (int*)c->list_a.p, counts + 0);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  k_screen<<<(unsigned)std::min<long long>(ncand, 8LL * std::max(nsm, 1)), 256, 0, c->stream>>>(
      (const double*)c->phi.p, n, c->N[0], c->N[1], c->N[2], (const int*)c->list_a.p, counts + 0,
      (const int*)c->cand_geom.p, c->dV, c->prm.delta, (int*)c->cand_flag.p,
      (double*)c->cand_S.p);
  k_compact<<<1, 1024, 0, c->stream>>>((const int*)c->cand_flag.p, 0, counts + 0,
                                       (int*)c->list_b.p, counts + 1);
  k_fill_pairs<<<gc, 256, 0, c->stream>>>((const int*)c->list_b.p, counts + 1,
                                          (const int*)c->list_a.p, (const int*)c->cand_geom.p,
                                          (const double*)c->cand_S.p, n, (PairInfo*)c->pinfo.p,
                                          (double*)c->pS.p, (int*)c->psize.p);
  k_scan_sizes<<<1, 1024, 0, c->stream>>>((const int*)c->psize.p, counts + 1,
                                          (const PairInfo*)c->pinfo.p, (long long*)c->voff.p,
                                          (long long*)(counts + 4), counts + 10);
  k_lpt_order<<<gc, 256, 0, c->stream>>>((const int*)c->psize.p, counts + 1, (int*)c->order.p);
  c->launches += 7;
  return cudaGetLastError();
}

}  // namespace sea
