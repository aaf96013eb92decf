// gram_tc.cu -- the mixed form's contraction with W on the tensor cores.
//
//   partial[s m + a] = sum over the points r of tile T of A[a][r] W[list(T)[s]][r]
//
// (s a slot of tile T's W list); the per-orbital sums of M = Phi^T W and of
// W^T psi add these partials afterwards in FP64.
//
// Precision: FP64 operands, FP64-accurate result from BF16 tensor-core
// products by exact splitting (the Ozaki scheme).  Each row segment x (the
// 64 points of one half tile, 8 x 4 x 2, of an A row or a W row) shares one
// exponent E (|x| < 2^E); x 2^-E is truncated to an integer X on a 2^-47
// grid and written in S = 6 balanced base-256 digits, x 2^-E ~ sum_k d_k
// 2^(-7-8k) with |d_k| <= 128, each exactly a BF16 value.  For a pair of
// segments,
//   sum_r x_r w_r ~ 2^(Ex+Ew) sum_{d=0}^{S-1} 2^(-14-8d) D_d,
//   D_d = sum_{k+l=d} sum_r dx_k(r) dw_l(r),
// where every D_d is a sum of at most 6 x 64 products of magnitude <= 2^14,
// hence an integer below 2^24: the tensor core's FP32 accumulation of it is
// exact.  The epilogue combines the D_d exactly in 64-bit integers; the
// per-thread-load kernel rounds each half tile once to FP64 and adds the
// two halves, the TMA kernel aligns the two halves' integers on the larger
// scale (the other truncated at its unit, 2^-54 of that segment's scale)
// and truncates once to FP64, with no FP64 instruction.  Error: the truncation of X
// (2^-47 of the segment maximum) and the dropped diagonals d >= S (below
// 2^-45.7 of max|x| max|w| times the segment length).
//
// Kernel shape: persistent CTAs (one per SM) take tiles from a queue and
// walk units (W block of up to 32 slots, A block of 128 rows, half tile).
// Per unit the A digits go to shared memory in the tensor core's K-major
// layout without swizzle (8 x 16-byte core matrices; row groups 128 B
// apart, x-runs of 8 points one row-group stack apart).  W's digit planes
// of the block are stacked along N (plane l at rows l P, P = 16 or 32 the
// padded block width) and the accumulator of diagonal d sits at
// tensor-memory columns d P, so one MMA of A plane k against the stacked W
// planes 0..5-k (N = (6 - k) P) adds every product of plane k to the
// diagonals k..5 at once: 24 tcgen05.mma instructions (M = 128, K = 16) per
// unit.  After the second half tile the converting warps read the
// accumulators back with tcgen05.ld for the epilogue.  Two versions:
//   k_gram_tc_ldg  512 threads load the A rows themselves and form their
//                  digits in registers while the previous unit's MMAs run
//                  (issued by thread 0); used when the rows are not
//                  16-byte strided (odd nx) or A is unaligned;
//   k_gram_tc      A rows by TMA per K half, 16 converting warps and one
//                  MMA-issuing warp (described above the kernel).
// Every wait on a completion barrier is bounded: on expiry the kernel sets
// SEA_FLAG_WAIT, waits once more (bounded) for work in flight, frees its
// tensor memory and ends.
#include <cuda.h>

#include "sea_internal.cuh"
#include "tcgen05.cuh"

namespace sea {
namespace {

constexpr int DIG = 6;                          // digits per operand
constexpr int KH = 64;                          // points per half tile
constexpr int NBLK = 32;                        // W rows per block
constexpr int MBLK = 128;                       // A rows per block
constexpr int GT_THREADS = 512;
constexpr uint32_t A_PLANE = MBLK * KH * 2;     // bytes per digit plane of A
constexpr uint32_t W_HALF = DIG * NBLK * KH * 2;  // bytes of W digits per half tile
constexpr uint32_t A_LBO = (MBLK / 8) * 128;    // K-adjacent core matrices of A
constexpr uint32_t CORE_SBO = 128;              // row-group-adjacent core matrices
constexpr uint32_t SMEM_A = DIG * A_PLANE;      // 96 KB
constexpr uint32_t SMEM_W = 2 * W_HALF;         // 48 KB (both halves)
constexpr size_t GT_SMEM = SMEM_A + 2 * SMEM_W + 128;  // A digits, two W buffers
constexpr uint32_t TMEM_HALF = DIG * NBLK;      // accumulator columns per half tile
constexpr uint32_t TMEM_COLS = 512;             // 2 x 192 columns used
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// x 2^-E on the 2^-47 grid (truncated toward zero), E = emax - 1022 for
// the segment's largest biased exponent emax: a signed integer below 2^47.
// Integer operations only.
__device__ __forceinline__ long long fixed47(double v, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const int sh = emax - e + 6;
  if (e == 0 || sh > 60) return 0;
  const long long X = (long long)(((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52)) >> sh);
  return (b >> 63) ? -X : X;
}

// Balanced base-256 digits of X: with Y = X + 128 (256^0 + ... + 256^4),
// digit 5 - i = byte i of Y minus 128 (i < 5) and digit 0 = Y >> 40, so
// X = sum_k d_k 256^(5-k), d_1..d_5 in [-128, 127], |d_0| <= 128.  Each
// digit as an FP32 value (exact), from the bit pattern 0x4B4000bb = 2^23 +
// 2^22 + b.
__device__ __forceinline__ void digit_floats(long long X, float* f) {
  const long long Y = X + 0x8080808080LL;
  const unsigned lo = (unsigned)Y, hi = (unsigned)(Y >> 32);
  const float m = 12582912.0f + 128.0f;
  f[5] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7650)) - m;
  f[4] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7651)) - m;
  f[3] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7652)) - m;
  f[2] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7653)) - m;
  f[1] = __uint_as_float(__byte_perm(hi, 0x4B400000u, 0x7650)) - m;
  f[0] = __int_as_float(0x4B400000 + (int)(Y >> 40)) - 12582912.0f;
}

// BF16 bit patterns of two small integer-valued floats, packed low/high.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// FP16 bit patterns of two small integer-valued floats (|v| <= 2048, exact),
// packed low/high.
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Digits of one row group (8 rows) of a block, half h of tile T, held in
// registers: the warp's lane l takes row l % 8 and the x-runs u = l / 8 and
// l / 8 + 4 (run u: y = u % 4, z = 2h + u / 4, 8 points along x).  Row
// pointer rp (nullptr: zero row).
struct GroupDigits {
  uint32_t w[2][DIG][4];  // [run][digit plane][pair of points]
  int emax;               // the row's largest biased exponent
};

__device__ __forceinline__ void make_digits(const double* __restrict__ rp, const TileGeom& G,
                                            int T, int h, GroupDigits& o) {
  const int lane = threadIdx.x & 31;
  const int txi = T % G.ntx, tyi = (T / G.ntx) % G.nty, tzi = T / (G.ntx * G.nty);
  const int gx0 = txi * TX;
  double v[2][8];
  int em = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int u = (lane >> 3) + 4 * q;
    const int gy = tyi * TY + (u & 3), gz = tzi * TZ + 2 * h + (u >> 2);
    const bool in = rp && gy < G.ny && gz < G.nz;
    const double* src = in ? rp + ((size_t)gz * G.ny + gy) * G.nx + gx0 : rp;
    if (in && gx0 + 8 <= G.nx && (((uintptr_t)src) & 15) == 0) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(src) + p);
        v[q][2 * p] = t.x;
        v[q][2 * p + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int x = 0; x < 8; ++x) v[q][x] = (in && gx0 + x < G.nx) ? src[x] : 0.0;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x)
      em = max(em, (int)((__double_as_longlong(v[q][x]) >> 52) & 0x7FF));
  }
  em = max(em, __shfl_xor_sync(0xffffffffu, em, 8));
  em = max(em, __shfl_xor_sync(0xffffffffu, em, 16));
  o.emax = em;
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float f0[DIG], f1[DIG];
      digit_floats(fixed47(v[q][2 * p], em), f0);
      digit_floats(fixed47(v[q][2 * p + 1], em), f1);
#pragma unroll
      for (int k = 0; k < DIG; ++k) o.w[q][k][p] = pack_f16(f0[k], f1[k]);
    }
}

// Digit planes of the group to shared memory (core matrices: row group g
// 128 B apart, run u one lbo apart, row l % 8 at 16 B), and the exponent
// (lanes 0..7) to emax_row[l % 8].
__device__ __forceinline__ void store_digits(const GroupDigits& o, unsigned char* plane0,
                                             uint32_t plane_bytes, uint32_t lbo, int g,
                                             int* emax_row) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    unsigned char* dst = plane0 + g * CORE_SBO + ((lane >> 3) + 4 * q) * lbo + (lane & 7) * 16;
#pragma unroll
    for (int k = 0; k < DIG; ++k)
      *reinterpret_cast<uint4*>(dst + k * plane_bytes) =
          make_uint4(o.w[q][k][0], o.w[q][k][1], o.w[q][k][2], o.w[q][k][3]);
  }
  if (lane < 8) emax_row[lane] = o.emax;
}

// Integer value of an integer-valued FP32 number at most 2^22 in magnitude:
// adding 1.5 2^23 puts it in the low mantissa bits.
__device__ __forceinline__ int small_float_int(uint32_t f) {
  return __float_as_int(__uint_as_float(f) + 12582912.0f) - 0x4B400000;
}

// v 2^e2 truncated toward zero to FP64, 0 below the normal range: the same
// value as scaled_i64_rz, with the 64-bit truncating conversion done by the
// conversion instruction (on the FP64 pipe, which the integer epilogues
// otherwise leave idle) and the scaling by 2^e2 added to the exponent field.
__device__ __forceinline__ double scaled_i64_rz_cvt(long long v, int e2) {
  const long long b = __double_as_longlong(__ll2double_rz(v));
  const int ex = (int)((b >> 52) & 0x7FF) + e2;  // biased exponent of the result
  return (v == 0 || ex <= 0) ? 0.0 : __longlong_as_double(b + ((long long)e2 << 52));
}

// Exact value of an integer-valued float below 2^24 in magnitude.
__device__ __forceinline__ int float_int(float f) {
  const unsigned u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 255);
  if (e < 127) return 0;
  const int mag = (int)(((u & 0x7FFFFFu) | 0x800000u) >> (150 - e));
  return (u >> 31) ? -mag : mag;
}


// W digits, once per W: for every slot s of every tile list and half h,
// wdig[((s * 2 + h) * DIG + k) * 8 + u] = the 8 BF16 digits (16 bytes) of
// plane k, x-run u of W row list[s] on that half tile, and wexp[2 s + h]
// the row segment's largest biased exponent.  Warp per (tile, half, group
// of 8 slots).  Four CTAs per SM: the warps wait on their row loads, so
// occupancy is what hides the latency.
__global__ void __launch_bounds__(256, 4)
    k_w_digits(const double* __restrict__ W, TileGeom G, size_t ng, int n_tiles, int ngroups,
               const int* __restrict__ tptr, const int* __restrict__ tlist, uint4* __restrict__ wdig,
               int* __restrict__ wexp) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (long long)n_tiles * 2 * ngroups) return;  // warp-uniform
  const int g = (int)(gw % ngroups), h = (int)((gw / ngroups) % 2), T = (int)(gw / (2 * ngroups));
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (8 * g >= nJ) return;  // warp-uniform
  const int lane = threadIdx.x & 31, r = lane & 7, s = 8 * g + r;
  const double* rp = s < nJ ? W + (size_t)tlist[j0 + s] * ng : nullptr;
  GroupDigits d;
  make_digits(rp, G, T, h, d);
  if (s < nJ) {
    uint4* dst = wdig + ((size_t)(j0 + s) * 2 + h) * DIG * 8;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int u = (lane >> 3) + 4 * q;
#pragma unroll
      for (int k = 0; k < DIG; ++k) dst[k * 8 + u] = make_uint4(d.w[q][k][0], d.w[q][k][1], d.w[q][k][2], d.w[q][k][3]);
    }
    if (lane < 8) wexp[(size_t)(j0 + s) * 2 + h] = d.emax;
  }
}

// A unit of work: half h of A block mb against W block jb of tile T, whose
// W digits are in buffer wb.
struct Unit {
  int T, j0, nJ, jb, mb, h, wb;
  int ab;  // parity of the A block in processing order (TMA kernel: its exponent buffer)
};


__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gram_tc_ldg(const double* __restrict__ A, int m, TileGeom G, size_t ng, int n_tiles,
              const int* __restrict__ tptr, const uint4* __restrict__ wdig,
              const int* __restrict__ wexp, double* __restrict__ partial, int* __restrict__ queue,
              unsigned* __restrict__ status) {
  extern __shared__ unsigned char gt_raw[];
  unsigned char* sA = gt_raw + ((128 - (smem_addr(gt_raw) & 127)) & 127);
  unsigned char* sW = sA + SMEM_A;  // two buffers of SMEM_W
  __shared__ int Aexp[2][MBLK], Wexp[2][2][NBLK];  // [half][row], [buffer][half][row]
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_tile, s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar = smem_addr(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t a_base = smem_addr(sA), w_base = smem_addr(sW);
  const int nmb = (m + MBLK - 1) / MBLK;

  // first unit of the next tile with a non-empty list; uniform, contains
  // __syncthreads (false: no tile left)
  auto claim = [&](Unit& u) -> bool {
    __syncthreads();
    if (tid == 0) {
      int t;
      do {
        t = atomicAdd(queue, 1);
      } while (t < n_tiles && tptr[t + 1] == tptr[t]);
      s_tile = t;
    }
    __syncthreads();
    const int T = s_tile;
    if (T >= n_tiles) return false;
    u.T = T;
    u.j0 = tptr[T];
    u.nJ = tptr[T + 1] - u.j0;
    u.jb = 0;
    u.mb = 0;
    u.h = 0;
    u.wb ^= 1;
    return true;
  };
  // the unit after u; *new_block: it starts another W block
  auto advance = [&](Unit& u, bool* new_block) -> bool {
    *new_block = false;
    if (u.h == 0) {
      u.h = 1;
      return true;
    }
    u.h = 0;
    if (++u.mb < nmb) return true;
    u.mb = 0;
    *new_block = true;
    u.jb += NBLK;
    if (u.jb < u.nJ) {
      u.wb ^= 1;
      return true;
    }
    return claim(u);
  };
  auto a_row = [&](const Unit& u) -> const double* {
    const int a = u.mb * MBLK + 8 * warp + (lane & 7);
    return a < m ? A + (size_t)a * ng : nullptr;
  };
  // W digits of u's block (both halves) into buffer u.wb, planes stacked
  // along N with row stride P (16 or 32): row l P + slot of half h at core
  // matrix (row / 8, run), K-adjacent ones 6 P 16 bytes apart.  16-byte
  // asynchronous copies, zeros beyond the list (completed before the next
  // __syncthreads that precedes the MMAs reading them).
  auto load_w = [&](const Unit& u) {
    const int nj = min(NBLK, u.nJ - u.jb), P = nj <= 16 ? 16 : 32;
    const uint32_t lbo = DIG * P * 16;
    const uint32_t dst0 = w_base + u.wb * SMEM_W;
    for (int p = tid; p < P * 2 * DIG * 8; p += GT_THREADS) {
      const int run = p & 7, k = (p >> 3) % DIG, h = (p / (8 * DIG)) & 1, sl = p / (16 * DIG);
      const bool ok = sl < nj;
      const uint4* src = ok ? wdig + ((size_t)(u.j0 + u.jb + sl) * 2 + h) * DIG * 8 + k * 8 + run : wdig;
      const int row = k * P + sl;
      cp_async16(dst0 + h * W_HALF + (row >> 3) * CORE_SBO + run * lbo + (row & 7) * 16, src, ok);
    }
    if (tid < 2 * NBLK) {
      const int h = tid / NBLK, sl = tid % NBLK;
      Wexp[u.wb][h][sl] = sl < nj ? wexp[(size_t)(u.j0 + u.jb + sl) * 2 + h] : 0;
    }
  };
  // partials of u's A block (both halves done): warp = (lane quarter q,
  // column class g), columns g, g + 4, ... of the block
  auto epilogue = [&](const Unit& u) {
    const int nj = min(NBLK, u.nJ - u.jb), P = nj <= 16 ? 16 : 32;
    const int quarter = warp & 3, g = warp >> 2;
    const int a = u.mb * MBLK + 32 * quarter + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
    const int ea0 = Aexp[0][32 * quarter + lane] - 1022, ea1 = Aexp[1][32 * quarter + lane] - 1022;
#pragma unroll 1
    for (int c = g; c < nj; c += 4) {
      uint32_t f[2 * DIG];
#pragma unroll
      for (int q = 0; q < 2 * DIG; ++q)
        f[q] = tmem_ld1(lane_addr + (uint32_t)((q / DIG) * TMEM_HALF + (q % DIG) * P + c));
      tmem_wait_ld();
      double sum = 0.0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        long long acc = 0;
#pragma unroll
        for (int d = 0; d < DIG; ++d)
          acc += (long long)float_int(__uint_as_float(f[h * DIG + d])) << (8 * (DIG - 1 - d));
        sum += scaled_i64(acc, (h ? ea1 : ea0) + (Wexp[u.wb][h][c] - 1022) - 54);
      }
      if (a < m) partial[(size_t)(u.j0 + u.jb + c) * m + a] = sum;
    }
  };
  // the MMAs of unit u (half u.h), then the commit: for K step q and A
  // plane k, one MMA against W planes 0..5-k into diagonals k..5
  auto issue = [&](const Unit& u) {
    const int nj = min(NBLK, u.nJ - u.jb), P = nj <= 16 ? 16 : 32;
    const uint32_t lbo = DIG * P * 16;
    // descriptors differ only in the start address (low 14 bits, no
    // carry: shared addresses are below 2^18)
    const uint64_t a0 = sdesc(a_base, A_LBO, CORE_SBO);
    const uint64_t w0 = sdesc(w_base + u.wb * SMEM_W + u.h * W_HALF, lbo, CORE_SBO);
    const uint32_t dcol = tmem + (uint32_t)(u.h * TMEM_HALF);
#pragma unroll
    for (int q = 0; q < KH / 16; ++q)
#pragma unroll
      for (int k = 0; k < DIG; ++k)
        mma_kf16(dcol + (uint32_t)(k * P), a0 + ((k * A_PLANE + q * 2 * A_LBO) >> 4),
                 w0 + ((q * 2 * lbo) >> 4), idesc_kf16((DIG - k) * P, MBLK, false), (k > 0 || q > 0) ? 1u : 0u);
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
  };

  Unit cur;
  cur.wb = 1;
  if (claim(cur)) {
    load_w(cur);
    GroupDigits dg;
    make_digits(a_row(cur), G, cur.T, cur.h, dg);
    Unit prev = cur;
    bool have_prev = false;
    uint32_t phase = 0;
    for (;;) {
      if (have_prev) {
        // prev's MMAs done: the A digits and the accumulators are free
        const bool ok = mbar_wait(bar, phase);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        phase ^= 1;
        tc_fence_after();
        if (prev.h == 1) {
          epilogue(prev);
          __syncthreads();  // the exponents are read before they are replaced
        }
      }
      store_digits(dg, sA, A_PLANE, A_LBO, warp, &Aexp[cur.h][8 * warp]);
      cp_async_wait_all();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) issue(cur);
      prev = cur;
      have_prev = true;
      // while the MMAs run: the next unit's W digits (a new block goes to
      // the other buffer, whose MMAs are done) and A digits
      bool new_block;
      if (!advance(cur, &new_block)) break;
      if (new_block) load_w(cur);
      make_digits(a_row(cur), G, cur.T, cur.h, dg);
    }
    // the last unit: its MMAs (bounded wait) and epilogue
    if (!s_fail) {
      const bool ok = mbar_wait(bar, phase);
      if (!ok) s_fail = 1;
      __syncthreads();
      if (!s_fail) {
        tc_fence_after();
        if (prev.h == 1) epilogue(prev);
      }
    }
    if (s_fail) mbar_wait(bar, phase);  // once more, bounded, before freeing
  }
  cp_async_wait_all();
  if (s_fail && tid == 0) atomicOr(status, SEA_FLAG_WAIT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// The same contraction with A's rows brought in by the tensor memory
// accelerator.  Per unit two 4D boxes (x 8, y 4, z 1, rows 128): the two
// z-planes of the half tile (K halves 0 and 1) for the whole A block, 32 KB
// each, written with the 64-byte swizzle so that the reads below are free
// of bank conflicts.  Thread t takes row t / 4 and the x-run y = t % 4 of
// both planes (16 values; the row's exponent from a 4-lane maximum), forms
// the digits in registers and stores one 16-byte core-matrix row per digit
// plane.  The MMAs of K half 0 (committed to barrier 0) run while K half 1
// is converted; those of K half 1 (barrier 1) run while the next unit's
// rows are read and converted.  Both raw buffers are refilled for the next
// unit as soon as their values are in registers.  Points outside the grid
// and rows beyond m read the box's zero fill.  One W buffer: a new W block
// is loaded after every MMA of the previous block completed.
// ---------------------------------------------------------------------------
constexpr int GT2_CONV = 512;                        // converting threads: 4 per A row
constexpr int GT2_THREADS = GT2_CONV + 32;           // and one MMA-issuing warp
constexpr uint32_t A2_LBO = (MBLK / 8) * 128 + 32;   // 2080: x-runs 8 banks apart
constexpr uint32_t A2_PLANE = 8 * A2_LBO;            // 8 runs of 8 points
constexpr uint32_t SMEM_A2 = DIG * A2_PLANE;         // 99,840
constexpr uint32_t RAW_KHALF = MBLK * (KH / 2) * 8;  // 32 KB: 128 rows x 32 points
constexpr size_t GT2_SMEM = 1024 + 2 * RAW_KHALF + SMEM_A2 + SMEM_W;

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// L2 prefetch of bytes (a multiple of 16) at p (16-byte aligned).
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// A's digits in the TMA kernel: unsigned bytes of |x| on the segment's
// 2^-48 grid, each carrying the sign of x.  With E = emax - 1022 (|x| <
// 2^E), X = floor(|x| 2^(48 - E)) = m >> (emax - e + 5) for the 53-bit
// significand m and biased exponent e of x, so X < 2^48 and
//   x ~ s 2^(E - 48) sum_k b_k 256^(5 - k),  b_k = byte 5 - k of X,
// with an error below 2^(E - 48).  b_k in [0, 255] is exact in FP16; the
// FP16 pattern 0x6400 | b is 1024 + b, so one packed FMA (1024 + b) s -
// 1024 s gives the signed digit s b for two points at once.  Against W's
// balanced digits (|d| <= 128) every product is below 2^15 and a diagonal
// sum of at most 6 x 64 of them stays below 2^24, exact in the FP32
// accumulator.  em_sh = (emax + 5) << 20; segments whose largest value is
// below 2^-959 (emax < 64) are taken as zero (em_sh = 0xF0000000 makes
// every shift reach 64).  Integer work per value: the exponent field, the
// shift count, the significand word, one 64-bit shift; per pair of values
// nine byte permutations and the sign word.

// 64-bit right shift, the count clamped at 64 (shr.b64 semantics).
__device__ __forceinline__ unsigned long long shr64(unsigned long long a, uint32_t n) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(n));
  return r;
}

__device__ __forceinline__ uint32_t hfma2_u(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// X of one value: the significand of v (bits h, l) shifted onto the grid.
__device__ __forceinline__ unsigned long long fixed48(uint32_t h, uint32_t l, uint32_t em_sh) {
  const uint32_t sh = (em_sh - (h & 0x7FF00000u)) >> 20;
  const unsigned long long m = ((unsigned long long)((h & 0xFFFFFu) | 0x100000u) << 32) | l;
  return shr64(m, sh);
}

// The six FP16 digit planes of 8 consecutive points: d[k] = their 8 signed
// digits of plane k (points 2i, 2i + 1 in word i, low half first).
__device__ __forceinline__ void digits8_u(const double (&v)[8], uint32_t em_sh, uint4 (&d)[DIG]) {
  constexpr uint32_t K64 = 0x64646464u;
  uint32_t w[DIG][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(v[2 * i]);
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(v[2 * i + 1]);
    const uint32_t h0 = (uint32_t)(b0 >> 32), h1 = (uint32_t)(b1 >> 32);
    const unsigned long long X0 = fixed48(h0, (uint32_t)b0, em_sh);
    const unsigned long long X1 = fixed48(h1, (uint32_t)b1, em_sh);
    const uint32_t x0h = (uint32_t)(X0 >> 32), x0l = (uint32_t)X0;
    const uint32_t x1h = (uint32_t)(X1 >> 32), x1l = (uint32_t)X1;
    // bytes of the two points interleaved: [p0 b, p1 b, p0 b', p1 b']
    const uint32_t tH = __byte_perm(x0h, x1h, 0x5140);  // bytes 4, 5 of X
    const uint32_t tB = __byte_perm(x0l, x1l, 0x7362);  // bytes 2, 3
    const uint32_t tA = __byte_perm(x0l, x1l, 0x5140);  // bytes 0, 1
    // sign word: FP16 pair (s0, s1) = +-1, and -1024 (s0, s1)
    const uint32_t S = (__byte_perm(h0, h1, 0x7030) & 0x80008000u) | 0x3C003C00u;
    const uint32_t C = S ^ 0xD800D800u;
    // plane k = byte 5 - k: FP16 1024 + b from the pattern 0x64bb
    w[0][i] = hfma2_u(__byte_perm(tH, K64, 0x4342), S, C);
    w[1][i] = hfma2_u(__byte_perm(tH, K64, 0x4140), S, C);
    w[2][i] = hfma2_u(__byte_perm(tB, K64, 0x4342), S, C);
    w[3][i] = hfma2_u(__byte_perm(tB, K64, 0x4140), S, C);
    w[4][i] = hfma2_u(__byte_perm(tA, K64, 0x4342), S, C);
    w[5][i] = hfma2_u(__byte_perm(tA, K64, 0x4140), S, C);
  }
#pragma unroll
  for (int k = 0; k < DIG; ++k) d[k] = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
}

// The same unsigned-byte FP16 digits for a pair of values with exponents of
// their own (the expansion's H(j, v) 2^E_j against E_v): emax0, emax1 are
// the largest biased exponents the two values are measured against (below 64:
// the value counts as zero).  pk[k][e] = the pair's digits of plane k.
__device__ __forceinline__ void digits2_u(double v0, double v1, int emax0, int emax1,
                                          uint32_t (&pk)[DIG][2], int e) {
  constexpr uint32_t K64 = 0x64646464u;
  const uint32_t em0 = emax0 >= 64 ? (uint32_t)(emax0 + 5) << 20 : 0xF0000000u;
  const uint32_t em1 = emax1 >= 64 ? (uint32_t)(emax1 + 5) << 20 : 0xF0000000u;
  const unsigned long long b0 = (unsigned long long)__double_as_longlong(v0);
  const unsigned long long b1 = (unsigned long long)__double_as_longlong(v1);
  const uint32_t h0 = (uint32_t)(b0 >> 32), h1 = (uint32_t)(b1 >> 32);
  const unsigned long long X0 = fixed48(h0, (uint32_t)b0, em0);
  const unsigned long long X1 = fixed48(h1, (uint32_t)b1, em1);
  const uint32_t x0h = (uint32_t)(X0 >> 32), x0l = (uint32_t)X0;
  const uint32_t x1h = (uint32_t)(X1 >> 32), x1l = (uint32_t)X1;
  const uint32_t tH = __byte_perm(x0h, x1h, 0x5140);
  const uint32_t tB = __byte_perm(x0l, x1l, 0x7362);
  const uint32_t tA = __byte_perm(x0l, x1l, 0x5140);
  const uint32_t S = (__byte_perm(h0, h1, 0x7030) & 0x80008000u) | 0x3C003C00u;
  const uint32_t C = S ^ 0xD800D800u;
  pk[0][e] = hfma2_u(__byte_perm(tH, K64, 0x4342), S, C);
  pk[1][e] = hfma2_u(__byte_perm(tH, K64, 0x4140), S, C);
  pk[2][e] = hfma2_u(__byte_perm(tB, K64, 0x4342), S, C);
  pk[3][e] = hfma2_u(__byte_perm(tB, K64, 0x4140), S, C);
  pk[4][e] = hfma2_u(__byte_perm(tA, K64, 0x4342), S, C);
  pk[5][e] = hfma2_u(__byte_perm(tA, K64, 0x4140), S, C);
}

// Converting warps 0..15 (named barrier 1) and the issuing warp 16.  Per
// unit the converting warps post the unit's block width and half to a
// two-entry ring and arrive on ready[0] once K half 0's digits are in place,
// on ready[1] once K half 1's are; the issuing thread waits on each,
// issues that K half's MMAs and commits them to mma[0] / mma[1].  A unit
// with width 0 ends the issuing loop.
__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }
// The same barrier returning whether v held in any converting thread (the
// same value in all of them).
__device__ __forceinline__ bool conv_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, 512, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(GT2_THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmA, int m, TileGeom G, int n_tiles,
              const int* __restrict__ tptr, const uint4* __restrict__ wdig,
              const int* __restrict__ wexp, double* __restrict__ partial, int* __restrict__ queue,
              unsigned* __restrict__ status) {
  extern __shared__ unsigned char gt_raw[];
  unsigned char* sR = gt_raw + ((1024 - (smem_addr(gt_raw) & 1023)) & 1023);  // two K halves
  unsigned char* sA = sR + 2 * RAW_KHALF;
  unsigned char* sW = sA + SMEM_A2;
  __shared__ int Aexp[2][2][MBLK], Wexp[2][2][NBLK];  // [A block parity][half][row],
                                                     // [W block parity][half][slot]
  __shared__ __align__(8) unsigned long long mbar[2], tbar[2], rbar[2];
  __shared__ int u_ring[2][2];  // per posted unit: W block width (0: end), half
  __shared__ uint32_t tmem_base;
  __shared__ int s_tile, s_j[2], s_fail, s_ifail;  // claimed tile, its list bounds; failures
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t mb[2] = {smem_addr(&mbar[0]), smem_addr(&mbar[1])};
  const uint32_t tb[2] = {smem_addr(&tbar[0]), smem_addr(&tbar[1])};
  const uint32_t rb[2] = {smem_addr(&rbar[0]), smem_addr(&rbar[1])};

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb[q]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tb[q]));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(rb[q]));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    s_fail = 0;
    s_ifail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t a_base = smem_addr(sA), w_base = smem_addr(sW), r_base = smem_addr(sR);

  if (warp == GT2_CONV / 32) {
    // ---- the issuing warp ----
    if (lane == 0) {
      uint32_t rph[2] = {0, 0};
      for (int seq = 0;; ++seq) {
        if (!mbar_wait(rb[0], rph[0])) {
          s_ifail = 1;
          break;
        }
        rph[0] ^= 1;
        const int nj = u_ring[seq & 1][0], h = u_ring[seq & 1][1];
        if (nj == 0) break;
        const int P = nj <= 16 ? 16 : 32;
        const uint32_t lbo = DIG * P * 16;
        const uint64_t a0 = sdesc(a_base, A2_LBO, CORE_SBO);
        const uint64_t w0 = sdesc(w_base + h * W_HALF, lbo, CORE_SBO);
        const uint32_t dcol = tmem + (uint32_t)(h * TMEM_HALF);
        for (int kh = 0; kh < 2; ++kh) {
          if (kh == 1) {
            if (!mbar_wait(rb[1], rph[1])) {
              s_ifail = 1;
              break;
            }
            rph[1] ^= 1;
          }
          tc_fence_after();
#pragma unroll
          for (int qq = 0; qq < 2; ++qq) {
            const int q = 2 * kh + qq;
#pragma unroll
            for (int k = 0; k < DIG; ++k)
              mma_kf16(dcol + (uint32_t)(k * P), a0 + ((k * A2_PLANE + q * 2 * A2_LBO) >> 4),
                       w0 + ((q * 2 * lbo) >> 4), idesc_kf16((DIG - k) * P, MBLK, false),
                       (k > 0 || q > 0) ? 1u : 0u);
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  mb[kh])
              : "memory");
        }
        if (s_ifail) break;
      }
    }
    __syncwarp();
  } else {
    // ---- the converting warps ----
    const int nmb = (m + MBLK - 1) / MBLK;
    // the thread that issues the A rows' TMA loads (lane 0 of the last
    // converting warp: thread 0 already claims the tiles)
    constexpr int TMA_TID = GT2_CONV - 32;
    bool tma_pending[2] = {false, false};  // meaningful in TMA_TID
    // this thread's row and x-run, and the swizzled offset of its run
    const int row = tid >> 2, run = tid & 3;
    const uint32_t r_off = (uint32_t)(row * 256 + run * 64);
    const uint32_t r_swz = (uint32_t)((((row & 1) << 1) | (run >> 1)) << 4);
    // Thread 0 claims tiles one ahead: the next index is taken from the
    // queue when the current tile is published, and over the following units
    // its bounds are read (q_stage 1 -> 2), empty tiles skipped and its first
    // W block prefetched to L2 (2 -> 3), so a claim seldom waits on memory.
    int q_t = 0, q_j0 = 0, q_j1 = 0, q_stage = 0;  // 1 index taken, 2 bounds read, 3 resolved
    auto q_step = [&]() {
      if (q_stage == 1) {
        if (q_t < n_tiles) {
          q_j0 = __ldg(tptr + q_t);
          q_j1 = __ldg(tptr + q_t + 1);
          q_stage = 2;
        } else {
          q_stage = 3;
        }
      } else if (q_stage == 2) {
        if (q_j1 == q_j0) {
          q_t = atomicAdd(queue, 1);
          q_stage = 1;
        } else {
          bulk_prefetch_l2(wdig + (size_t)q_j0 * 2 * DIG * 8,
                           (uint32_t)min(q_j1 - q_j0, NBLK) * 2 * DIG * 8 * 16);
          q_stage = 3;
        }
      }
    };
    auto claim = [&](Unit& u) -> bool {
      conv_sync();
      if (tid == 0) {
        if (q_stage == 0) {
          q_t = atomicAdd(queue, 1);
          q_stage = 1;
        }
        while (q_stage != 3) q_step();
        s_tile = q_t;
        s_j[0] = q_j0;
        s_j[1] = q_j1;
        if (q_t < n_tiles) {
          q_t = atomicAdd(queue, 1);
          q_stage = 1;
        }
      }
      conv_sync();
      const int T = s_tile;
      if (T >= n_tiles) return false;
      u.T = T;
      u.j0 = s_j[0];
      u.nJ = s_j[1] - u.j0;
      u.jb = 0;
      u.mb = 0;
      u.h = 0;
      return true;
    };
    auto advance = [&](Unit& u, bool* new_block) -> bool {
      *new_block = false;
      if (u.h == 0) {
        u.h = 1;
        return true;
      }
      u.h = 0;
      u.ab ^= 1;
      if (++u.mb < nmb) return true;
      u.mb = 0;
      *new_block = true;
      u.wb ^= 1;
      u.jb += NBLK;
      if (u.jb < u.nJ) return true;
      return claim(u);
    };
    // K half q (z-plane 2 h + q of the half tile) of unit u's A block (thread 0)
    auto tma_issue = [&](const Unit& u, int q) {
      const int txi = u.T % G.ntx, tyi = (u.T / G.ntx) % G.nty, tzi = u.T / (G.ntx * G.nty);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(tb[q], RAW_KHALF);
      tma_load_4d(r_base + q * RAW_KHALF, &tmA, txi * TX, tyi * TY, tzi * TZ + 2 * u.h + q,
                  u.mb * MBLK, tb[q]);
      tma_pending[q] = true;
    };
    auto load_w = [&](const Unit& u) {
      const int nj = min(NBLK, u.nJ - u.jb), P = nj <= 16 ? 16 : 32;
      const uint32_t lbo = DIG * P * 16;
      for (int p = tid; p < P * 2 * DIG * 8; p += GT2_CONV) {
        const int rn = p & 7, k = (p >> 3) % DIG, h = (p / (8 * DIG)) & 1, sl = p / (16 * DIG);
        const bool ok = sl < nj;
        const uint4* src =
            ok ? wdig + ((size_t)(u.j0 + u.jb + sl) * 2 + h) * DIG * 8 + k * 8 + rn : wdig;
        const int r = k * P + sl;
        cp_async16(w_base + h * W_HALF + (r >> 3) * CORE_SBO + rn * lbo + (r & 7) * 16, src, ok);
      }
      if (tid < 2 * NBLK) {
        const int h = tid / NBLK, sl = tid % NBLK;
        Wexp[u.wb][h][sl] = sl < nj ? wexp[(size_t)(u.j0 + u.jb + sl) * 2 + h] : 0;
      }
    };
    // bounded waits; false on expiry
    uint32_t tphase[2] = {0, 0}, mphase[2] = {0, 0};
    bool mma_pend[2] = {false, false};
    auto wait_raw = [&](int q) -> bool {
      const bool ok = mbar_wait(tb[q], tphase[q]);
      tphase[q] ^= 1;
      if (tid == TMA_TID) tma_pending[q] = false;
      return ok;
    };
    auto wait_mma = [&](int q) -> bool {
      if (!mma_pend[q]) return true;
      if (!mbar_wait(mb[q], mphase[q])) return false;
      mphase[q] ^= 1;
      mma_pend[q] = false;
      return true;
    };
    // digits of K half q (x-run run + 4 q of the half tile) to shared memory
    auto store_digits = [&](const uint4 (&d)[DIG], int q) {
      unsigned char* dst = sA + (row >> 3) * CORE_SBO + (run + 4 * q) * A2_LBO + (row & 7) * 16;
#pragma unroll
      for (int k = 0; k < DIG; ++k) *reinterpret_cast<uint4*>(dst + k * A2_PLANE) = d[k];
    };
    auto epilogue = [&](const Unit& u) {
      const int nj = min(NBLK, u.nJ - u.jb), P = nj <= 16 ? 16 : 32;
      const int quarter = warp & 3, g = warp >> 2, ng4 = GT2_CONV / 128;
      const int a = u.mb * MBLK + 32 * quarter + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
      const int ea0 = Aexp[u.ab][0][32 * quarter + lane] - 1022,
                ea1 = Aexp[u.ab][1][32 * quarter + lane] - 1022;
      // column pairs (c0, c0 + 1), c0 = 2 g, 2 g + 8, ...: one two-column
      // tensor-memory load per diagonal and half
#pragma unroll 1
      for (int c0 = 2 * g; c0 < nj; c0 += 2 * ng4) {
        // |D_d| < (d + 1) 2^21 (A digits up to 255, W digits up to 128 in
        // magnitude, 64 points): D_0, D_1 (< 2^22) by the 2^22 conversion on
        // the FP32 pipe, the others by the conversion unit (exact: integer
        // values below 2^24); D_0 256 + D_1 and D_2 256 + D_3 stay below 2^31
        long long acc[2][2];  // [half][column]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t f[DIG][2];
#pragma unroll
          for (int d = 0; d < DIG; ++d)
            tmem_ld2(lane_addr + (uint32_t)(h * TMEM_HALF + d * P + c0), f[d]);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int t01 = small_float_int(f[0][cc]) * 256 + small_float_int(f[1][cc]);
            const int t23 = __float2int_rz(__uint_as_float(f[2][cc])) * 256 +
                            __float2int_rz(__uint_as_float(f[3][cc]));
            acc[h][cc] = ((long long)t01 << 32) + ((long long)t23 << 16) +
                         ((long long)__float2int_rz(__uint_as_float(f[4][cc])) << 8) +
                         (long long)__float2int_rz(__uint_as_float(f[5][cc]));
          }
        }
        // sum_r x w = 2^(E_x + E_w - 55) acc; the two halves on the larger
        // scale (the other truncated at its unit, 2^-55 of that segment's
        // scale), one truncation
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = c0 + cc;
          if (c < nj) {
            const int e0 = ea0 + Wexp[u.wb][0][c] - 1022 - 55, e1 = ea1 + Wexp[u.wb][1][c] - 1022 - 55;
            const bool b0 = e0 >= e1;
            const int sh = min(b0 ? e0 - e1 : e1 - e0, 63);
            const long long s2 = (b0 ? acc[0][cc] : acc[1][cc]) + ((b0 ? acc[1][cc] : acc[0][cc]) >> sh);
            if (a < m) partial[(size_t)(u.j0 + u.jb + c) * m + a] = scaled_i64_rz_cvt(s2, b0 ? e0 : e1);
          }
        }
      }
    };

    // post unit u (or the end, nj = 0) to the issuing thread: ring entry
    // seq & 1, then ready[0] (thread 0, after a converting-warp barrier)
    auto post = [&](int seq, int nj, int h) {
      if (tid == 0) {
        u_ring[seq & 1][0] = nj;
        u_ring[seq & 1][1] = h;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rb[0]) : "memory");
      }
    };

    Unit cur;
    cur.wb = 0;
    cur.ab = 0;
    bool have_prev = false, fail = false;  // fail: uniform over the converting threads
    Unit prev = cur;
    int seq = 0;
    // Per unit two barriers of the converting warps: B1 once every thread
    // holds its values (the raw buffers may be refilled), B2 once the digits
    // of both K halves, a new W block and the exponents are in place (both K
    // halves are then posted).  The digit buffers are guarded per thread by
    // the MMA completion barriers, the A exponents double-buffered by A block.
    if (claim(cur)) {
      load_w(cur);
      if (tid == TMA_TID) {
        tma_issue(cur, 0);
        tma_issue(cur, 1);
      }
      bool need_w = false;
      for (;;) {
        // both K halves of cur to registers; the row's exponent
        bool ok = wait_raw(0);
        ok = wait_raw(1) && ok;
        double v[2][8];
        uint32_t emf = 0;  // largest exponent field (high-word bits 20..30) of the row segment
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const double2 t = *reinterpret_cast<const double2*>(
                sR + q * RAW_KHALF + r_off + (((uint32_t)p << 4) ^ r_swz));
            v[q][2 * p] = t.x;
            v[q][2 * p + 1] = t.y;
            emf = max(emf, (uint32_t)__double2hiint(t.x) & 0x7FF00000u);
            emf = max(emf, (uint32_t)__double2hiint(t.y) & 0x7FF00000u);
          }
        emf = max(emf, __shfl_xor_sync(0xffffffffu, emf, 1));
        emf = max(emf, __shfl_xor_sync(0xffffffffu, emf, 2));
        const int em = (int)(emf >> 20);
        const uint32_t em_sh = em < 64 ? 0xF0000000u : emf + (5u << 20);
        if (tid == 0) q_step();
        if (conv_sync_or(!ok)) {  // B1: both raw buffers consumed
          fail = true;
          break;
        }
        Unit next = cur;
        bool new_block = false;
        const bool has_next = advance(next, &new_block);  // may claim (uniform, syncs)
        if (tid == TMA_TID && has_next) {
          tma_issue(next, 0);
          tma_issue(next, 1);
        }
        // each K half's digits replace those prev's MMAs of that half read
        uint4 d[DIG];
        ok = wait_mma(0);
        digits8_u(v[0], em_sh, d);
        store_digits(d, 0);
        ok = wait_mma(1) && ok;
        digits8_u(v[1], em_sh, d);
        store_digits(d, 1);
        tc_fence_after();
        if (have_prev && prev.h == 1) epilogue(prev);  // all of prev's MMAs are done
        // a new W block: the MMAs that read the old one are done (waited
        // above) and its exponents sit in the other buffer
        if (need_w) load_w(cur);
        if (run == 0) Aexp[cur.ab][cur.h][row] = em;
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        if (conv_sync_or(!ok)) {  // B2: digits, W and exponents in place
          fail = true;
          break;
        }
        post(seq, min(NBLK, cur.nJ - cur.jb), cur.h);
        if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rb[1]) : "memory");
        ++seq;
        mma_pend[0] = mma_pend[1] = true;
        prev = cur;
        have_prev = true;
        if (!has_next) break;
        need_w = new_block;
        cur = next;
      }
    }
    // the last unit's MMAs (bounded waits; the issuing thread has then taken
    // every posted unit), the end of the issuing loop, the last epilogue
    if (!fail) {
      bool ok = wait_mma(0);
      ok = wait_mma(1) && ok;
      fail = conv_sync_or(!ok);
    }
    post(seq, 0, 0);
    if (!fail) {
      tc_fence_after();
      if (have_prev && prev.h == 1) epilogue(prev);
    } else {
      // once more, bounded, before the tensor memory is freed
      for (int q = 0; q < 2; ++q)
        if (mma_pend[q]) mbar_wait(mb[q], mphase[q]);
      // loads still in flight land before the CTA's shared memory is released
      if (tid == TMA_TID)
        for (int q = 0; q < 2; ++q)
          if (tma_pending[q]) mbar_wait(tb[q], tphase[q]);
    }
    cp_async_wait_all();
    if (fail && tid == 0) s_fail = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && (s_fail || s_ifail)) atomicOr(status, SEA_FLAG_WAIT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// The mixed form's expansion y[v][r] = sign sum_j W[list(j)][r] H(j, v) on
// the tensor cores, per tile (M = the tile's 128 points, N = vectors, K =
// the tile's W list, at most XJ = 32 entries; longer lists go to the FP32
// kernel).  Scales: W's digits are taken per (tile, list entry j) with the
// exponent E_j of that W row on the tile (six balanced FP16 digits a_k,
// |a_k| <= 128, on the 2^-47 grid); H(j, v) is scaled exactly by 2^E_j and
// measured against one exponent E_v per (tile, vector v) over the list, its
// digits the unsigned bytes b_l of |H| 2^(E_j - E_v) on the 2^-48 grid with
// H's sign (as A's in the contraction), so
//   y = 2^(E_v) sum_d 2^(-15-8d) D_d,  D_d = sum_j sum_{k+l=d} a_k(j) b_l(j),
// E_j cancels and every D_d (at most 32 x 6 products of magnitude < 2^15)
// is an integer below 2^23, exact in the FP32 accumulator.  W's digits are
// formed once per W into a per-tile image in the K-major layout (two K steps
// of 16 list entries, six planes, 4 KB each); H's digits per chunk of 32
// vectors into a slot of a shared-memory ring with the six planes stacked
// along N, so one MMA of A plane k against planes 0..5-k adds plane k's
// products to diagonals k..5 (TMEM columns 32 d).  Two accumulator buffers
// of 192 columns: the MMAs of chunk c + 1 run while chunk c's epilogue reads
// its buffer back, and the digits of the following chunks are formed
// meanwhile by warps of their own.
// ---------------------------------------------------------------------------
constexpr int XJ = 32, XKS = 16, XN = 32;
constexpr uint32_t XA_BLOCK = MBLK * XKS * 2;          // 4 KB: one plane, one K step
constexpr uint32_t XA_LBO = (MBLK / 8) * 128;          // 2048
constexpr uint32_t XA_STEP = DIG * XA_BLOCK;           // 24 KB
constexpr uint32_t XA_TILE = 2 * XA_STEP;              // 48 KB
constexpr uint32_t XB_LBO = (DIG * XN / 8) * 128;      // 3072
constexpr uint32_t XB_CHUNK = 2 * XB_LBO;              // 6 KB: 192 rows x 16 K
constexpr uint32_t XT_COLS = DIG * XN;                 // 192

// W's digit image: CTA per tile (thread = point p), for tiles whose list has
// 1..XJ entries.  wx[T][(q 6 + k) 4096 + (p / 8) 128 + (jq / 8) 2048 +
// (p % 8) 16 + (jq % 8) 2] = digit k of W[list(16 q + jq)] at point p (zero
// outside the entry's sub-box and beyond the list), wxexp[slot] = E_j + 1022.
__global__ void __launch_bounds__(MBLK)
    k_wx_digits(const double* __restrict__ W, TileGeom G, size_t ng, int n_tiles,
                const int* __restrict__ tptr, const int* __restrict__ tlist,
                const int* __restrict__ tsub, uint4* __restrict__ wx, int* __restrict__ wxexp) {
  const int T = blockIdx.x;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (nJ == 0 || nJ > XJ) return;  // uniform
  __shared__ int emx[XJ];
  const int p = threadIdx.x;
  if (p < XJ) emx[p] = 0;
  const long long g = tile_point(G, T, p);
  const int pz = p / (TX * TY), py = (p / TX) % TY, px = p % TX;
  auto wval = [&](int jl) -> double {
    if (jl >= nJ || g < 0) return 0.0;
    const int sb = tsub[j0 + jl];
    const bool in = px >= (sb & 15) && px < ((sb >> 4) & 15) && py >= ((sb >> 8) & 15) &&
                    py < ((sb >> 12) & 15) && pz >= ((sb >> 16) & 15) && pz < ((sb >> 20) & 15);
    return in ? W[(size_t)tlist[j0 + jl] * ng + g] : 0.0;
  };
  __syncthreads();
  for (int jl = 0; jl < nJ; ++jl)
    atomicMax(&emx[jl], (int)((__double_as_longlong(wval(jl)) >> 52) & 0x7FF));
  __syncthreads();
  if (p < nJ) wxexp[j0 + p] = emx[p];
  const int nq = (nJ + XKS - 1) / XKS;
  unsigned char* base = reinterpret_cast<unsigned char*>(wx) + (size_t)T * XA_TILE;
  for (int grp = 0; grp < 2 * nq; ++grp) {  // 8 list entries at a time
    uint32_t pk[DIG][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const int jl = 8 * grp + e;
      float f0[DIG], f1[DIG];
      digit_floats(jl < nJ ? fixed47(wval(jl), emx[jl]) : 0, f0);
      digit_floats(jl + 1 < nJ ? fixed47(wval(jl + 1), emx[jl + 1]) : 0, f1);
#pragma unroll
      for (int k = 0; k < DIG; ++k) pk[k][e / 2] = pack_f16(f0[k], f1[k]);
    }
    const int q = grp >> 1, jj = grp & 1;
#pragma unroll
    for (int k = 0; k < DIG; ++k)
      *reinterpret_cast<uint4*>(base + (q * DIG + k) * XA_BLOCK + (p >> 3) * 128 + jj * XA_LBO +
                                (p & 7) * 16) = make_uint4(pk[k][0], pk[k][1], pk[k][2], pk[k][3]);
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}


// E_v of the expansion for every (tile, vector): the largest biased
// exponent of H(j, v) 2^(E_j) over the tile's list (0 where all are zero);
// thread = vector, grid y = tile.  Tiles with an empty list or more than XJ
// entries are skipped (not read).
__global__ void __launch_bounds__(128)
    k_expand_ev(const int* __restrict__ tptr, const int* __restrict__ tlist,
                const int* __restrict__ wxexp, const double* __restrict__ H, long long hj,
                long long hv, int m, int* __restrict__ ev) {
  const int T = blockIdx.y, v = blockIdx.x * 128 + threadIdx.x;
  const int j0 = tptr[T], nJ = tptr[T + 1] - j0;
  if (v >= m || nJ == 0 || nJ > XJ) return;
  int em = 0;
  for (int jl = 0; jl < nJ; ++jl) {
    const int e =
        (int)((__double_as_longlong(H[(long long)tlist[j0 + jl] * hj + (long long)v * hv]) >> 52) &
              0x7FF);
    if (e) em = max(em, e + wxexp[j0 + jl] - 1022);
  }
  ev[(size_t)T * m + v] = em;
}

constexpr int XE_WARPS = 16;                 // epilogue warps (tensor-memory read-back, stores)
constexpr int XP_WARPS = 8;                  // H-digit warps
constexpr int XE_ISSUER = XE_WARPS + XP_WARPS;           // the MMA-issuing warp
constexpr int XE_THREADS = 32 * (XE_ISSUER + 1);         // 800
constexpr int XR = 4;                                    // ring slots (chunks of XN vectors)
constexpr uint32_t XS_SLOT = 2 * XB_CHUNK;               // 12 KB: both K steps of one chunk
constexpr size_t XE_SMEM = 2 * XA_TILE + XR * XS_SLOT + 128;
constexpr int XF_FIRST = 1, XF_LAST = 2, XF_END = 4;    // slot flags

// Persistent CTAs (one per SM) over the tiles whose list has at most XJ
// entries, in three roles that run side by side.
//  * H-digit warps (XP_WARPS): claim the tiles, bring each tile's W digit
//    image in (bulk copy, two buffers), and for every chunk of XN = 32
//    vectors of the tile form E_v and H's digits into the next slot of a
//    ring of XR chunks, with the chunk's tile, first vector and E_v beside
//    it; a slot is refilled once its MMAs are done and the epilogue warps
//    have read its E_v.
//  * The issuing warp: per chunk, once its slot is full (and, at a tile's
//    first chunk, the tile's W image is in) and the accumulator buffer it
//    takes is free, the chunk's MMAs into one of two buffers of 192
//    tensor-memory columns, committed to that buffer's barrier, to the
//    slot's and, at a tile's last chunk, to the W image's.
//  * Epilogue warps (16): warp w reads tensor-memory lanes 32 (w % 4) back
//    for vectors 8 (w / 4) .. + 7 of each chunk, combines the diagonal sums
//    and stores the FP64 outputs; zero tiles (empty list) are stored as
//    zeros without MMAs.
// So the digits of the next chunks and the MMAs of the next chunk run while
// a chunk's outputs are being converted and stored.  H(j, v) = H[j hj + v
// hv]; out[v ng + r].  Every wait is bounded; on expiry the role stops, the
// others see s_fail (or expire themselves) and the kernel reports
// SEA_FLAG_WAIT after the MMAs and copies in flight are done.
__global__ void __launch_bounds__(XE_THREADS, 1)
    k_expand_tc(const uint4* __restrict__ wx, const int* __restrict__ wxexp, TileGeom G, size_t ng,
                int n_tiles, const int* __restrict__ tptr, const int* __restrict__ tlist,
                const double* __restrict__ H, long long hj, long long hv, int m, int negate,
                double* __restrict__ out, const int* __restrict__ evp, int* __restrict__ queue,
                unsigned* __restrict__ status) {
  extern __shared__ unsigned char xe_raw[];
  unsigned char* sA = xe_raw + ((128 - (smem_addr(xe_raw) & 127)) & 127);  // two tile images
  unsigned char* sS = sA + 2 * XA_TILE;                                     // XR chunk slots
  __shared__ int s_T[XR], s_nJ[XR], s_v0[XR], s_fl[XR], s_ab[XR];
  __shared__ __align__(16) int s_ev[XR][XN];
  __shared__ int p_lj[XJ], p_shj[XJ], p_tile;
  __shared__ __align__(8) unsigned long long bar_full[XR], bar_free[XR], bar_md[2], bar_tf[2],
      bar_a[2], bar_af[2], bar_fin;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < XR; ++q) {
      mbar_init(smem_addr(&bar_full[q]), XP_WARPS);
      mbar_init(smem_addr(&bar_free[q]), 1 + XE_WARPS);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_addr(&bar_md[q]), 1);
      mbar_init(smem_addr(&bar_tf[q]), XE_WARPS);
      mbar_init(smem_addr(&bar_a[q]), 1);
      mbar_init(smem_addr(&bar_af[q]), 1);
    }
    mbar_init(smem_addr(&bar_fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t a_base = smem_addr(sA), s_base = smem_addr(sS);
  const int nch = (m + XN - 1) / XN;  // chunks per tile

  if (warp >= XE_WARPS && warp < XE_ISSUER) {
    // ---- H-digit warps: lane = vector of the chunk, warp pw = list entries
    // jp pw .. jp pw + jp - 1 with jp = 2 nq (so every warp has work) ----
    const int pw = warp - XE_WARPS, ptid = tid - 32 * XE_WARPS;
    auto pbar = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(32 * XP_WARPS) : "memory"); };
    auto pbar_or = [&](bool v) -> bool {
      uint32_t r;
      asm volatile(
          "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\n"
          "selp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(r)
          : "r"((uint32_t)v), "n"(32 * XP_WARPS)
          : "memory");
      return r != 0;
    };
    int pseq = 0, tseq = 0;               // chunks published; tiles whose W image was loaded
    uint32_t a_pend = 0, a_par = 0;       // ptid 0, bit b: a load into image buffer b was
                                          // issued; the parity of its completion
    bool fail = false;
    for (;;) {
      if (ptid == 0) {
        int t;
        do {
          t = atomicAdd(queue, 1);
        } while (t < n_tiles && tptr[t + 1] - tptr[t] > XJ);
        p_tile = t;
      }
      pbar();
      const int T = p_tile;
      const bool end = T >= n_tiles;
      const int j0 = end ? 0 : tptr[T], nJ = end ? 0 : tptr[T + 1] - j0;
      const int nq = (nJ + XKS - 1) / XKS, ab = tseq & 1, jp = 2 * nq, jb = jp * pw;
      if (ptid < nJ) {
        p_lj[ptid] = tlist[j0 + ptid];
        p_shj[ptid] = wxexp[j0 + ptid] - 1022;
      }
      bool ok = true;
      if (ptid == 0 && nJ > 0) {
        // the image buffer is free once the MMAs of the tile two back are done
        if (tseq >= 2) ok = mbar_wait(smem_addr(&bar_af[ab]), (uint32_t)(((tseq - 2) >> 1) & 1));
        if (ok) {
          const uint32_t bytes = (uint32_t)nq * XA_STEP;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(smem_addr(&bar_a[ab]), bytes);
          bulk_load(a_base + ab * XA_TILE,
                    reinterpret_cast<const unsigned char*>(wx) + (size_t)T * XA_TILE, bytes,
                    smem_addr(&bar_a[ab]));
          a_pend |= 1u << ab;
          a_par = (a_par & ~(1u << ab)) | ((uint32_t)((tseq >> 1) & 1) << ab);
        }
      }
      if (pbar_or(!ok || s_fail)) {  // p_lj, p_shj visible
        fail = true;
        break;
      }
      // H(j, v) of this thread's entries for chunk c (sign folded in), zero
      // beyond the list and the vectors, and E_v of the chunk's vector
      auto load_h = [&](int c, double (&h)[4], int& ev) {
        const int v = c * XN + lane;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int jl = jb + i;
          h[i] = (i < jp && v < m && jl < nJ) ? H[(long long)p_lj[jl] * hj + (long long)v * hv] : 0.0;
          if (negate)  // the sign of y folded into H's digits (sign bit, exact)
            h[i] = __longlong_as_double(__double_as_longlong(h[i]) ^ (long long)0x8000000000000000ULL);
        }
        ev = v < m ? evp[(size_t)T * m + v] : 0;
      };
      // chunk c from the values in h (the next chunk's values are loaded into
      // hn meanwhile: two register sets used in turn, so nothing waits on
      // those loads before the next chunk).  The warps of this role do not
      // wait on one another here: each waits for the slot itself and
      // arrives on its full barrier; a warp whose wait expired (wfail) skips
      // the rest of the tile's chunks and the role stops at the tile's end.
      bool wfail = false;
      auto chunk = [&](int c, double (&h)[4], int ev, double (&hn)[4], int& evn) {
        const int slot = pseq % XR, use = pseq / XR;
        ++pseq;
        if (wfail) return;
        // the slot is free once its previous chunk's MMAs are done and its
        // E_v was read
        bool ok = true;
        if (lane == 0) {
          if (use >= 1) ok = mbar_wait(smem_addr(&bar_free[slot]), (uint32_t)((use - 1) & 1));
          ok = ok && !s_fail;
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) {  // the same decision in every lane
          wfail = true;
          return;
        }
        if (nJ > 0) {
          if (c + 1 < nch) load_h(c + 1, hn, evn);
          if (pw == 0) s_ev[slot][lane] = ev;
          uint32_t pk[DIG][2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int jl = jb + 2 * e;
            digits2_u(h[2 * e], h[2 * e + 1], jl < nJ ? ev - p_shj[jl] : 0,
                      jl + 1 < nJ ? ev - p_shj[jl + 1] : 0, pk, e);
          }
          // entries jb.. of K step jb / 16: core matrix (jb / 8) % 2, bytes
          // (jb % 8) 2 of its 16-byte rows
          unsigned char* dst = sS + slot * XS_SLOT + (jb >> 4) * XB_CHUNK +
                               ((jb >> 3) & 1) * XB_LBO + (jb & 7) * 2;
#pragma unroll
          for (int l = 0; l < DIG; ++l) {
            const int row = l * XN + lane;
            unsigned char* q = dst + (row >> 3) * 128 + (row & 7) * 16;
            if (jp == 4)
              *reinterpret_cast<uint2*>(q) = make_uint2(pk[l][0], pk[l][1]);
            else
              *reinterpret_cast<uint32_t*>(q) = pk[l][0];
          }
        }
        if (ptid == 0) {
          s_T[slot] = T;
          s_nJ[slot] = nJ;
          s_v0[slot] = c * XN;
          s_fl[slot] = end ? XF_END : ((c == 0 ? XF_FIRST : 0) | (c == nch - 1 ? XF_LAST : 0));
          s_ab[slot] = ab;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // digits -> tensor core
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar_full[slot])) : "memory");
      };
      double hA[4], hB[4];
      int eA = 0, eB = 0;
      if (nJ > 0) load_h(0, hA, eA);
      const int nc = end ? 1 : nch;
      for (int c = 0; c < nc; c += 2) {
        chunk(c, hA, eA, hB, eB);
        if (c + 1 < nc) chunk(c + 1, hB, eB, hA, eA);
      }
      fail = pbar_or(wfail);  // every thread is done with this tile's lists
      if (fail || end) break;
      if (nJ > 0) ++tseq;
    }
    // image loads in flight land before the shared memory is released
    if (ptid == 0)
      for (int b = 0; b < 2; ++b)
        if ((a_pend >> b) & 1u) mbar_wait(smem_addr(&bar_a[b]), (a_par >> b) & 1u);
    if (fail) s_fail = 1;
  } else if (warp == XE_ISSUER) {
    // ---- the issuing warp ----
    if (lane == 0) {
      bool fail = false;
      long long cgm = 0;  // chunks with MMAs so far
      int tcount = 0;     // tiles with MMAs started
      for (int seq = 0;; ++seq) {
        const int slot = seq % XR, use = seq / XR;
        if (s_fail || !mbar_wait(smem_addr(&bar_full[slot]), (uint32_t)(use & 1))) {
          fail = true;
          break;
        }
        const int fl = s_fl[slot], nJ = s_nJ[slot], ab = s_ab[slot];
        if (fl & XF_END) break;
        if (nJ == 0) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar_free[slot])) : "memory");
          continue;
        }
        if (fl & XF_FIRST) {
          if (!mbar_wait(smem_addr(&bar_a[ab]), (uint32_t)((tcount >> 1) & 1))) {
            fail = true;
            break;
          }
          ++tcount;
        }
        const int tb = (int)(cgm & 1);
        const long long u = cgm >> 1;
        if (u >= 1 && !mbar_wait(smem_addr(&bar_tf[tb]), (uint32_t)((u - 1) & 1))) {
          fail = true;
          break;
        }
        tc_fence_after();
        const int nq = (nJ + XKS - 1) / XKS;
        const uint32_t dcol = tmem + (uint32_t)(tb * XT_COLS);
        for (int qq = 0; qq < nq; ++qq)
#pragma unroll
          for (int k = 0; k < DIG; ++k) {
            const uint64_t a = sdesc(a_base + ab * XA_TILE + qq * XA_STEP + k * XA_BLOCK, XA_LBO, 128);
            const uint64_t b = sdesc(s_base + slot * XS_SLOT + qq * XB_CHUNK, XB_LBO, 128);
            mma_kf16(dcol + (uint32_t)(k * XN), a, b, idesc_kf16((DIG - k) * XN, MBLK, false),
                     (k > 0 || qq > 0) ? 1u : 0u);
          }
        mma_commit(smem_addr(&bar_md[tb]));
        mma_commit(smem_addr(&bar_free[slot]));
        if (fl & XF_LAST) mma_commit(smem_addr(&bar_af[ab]));
        ++cgm;
      }
      // every MMA issued is done before the tensor memory is freed
      mma_commit(smem_addr(&bar_fin));
      mbar_wait(smem_addr(&bar_fin), 0);
      if (fail) s_fail = 1;
    }
    __syncwarp();
  } else {
    // ---- epilogue warps ----
    const int p = 32 * (warp & 3) + lane;  // tensor-memory lane = point of the tile
    const int vv0 = 8 * (warp >> 2);
    const uint32_t lane_q = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)vv0;
    long long cgm = 0, g = -1;
    int lastT = -1;
    bool fail = false;
    for (int seq = 0;; ++seq) {
      const int slot = seq % XR, use = seq / XR;
      bool ok = !s_fail && mbar_wait(smem_addr(&bar_full[slot]), (uint32_t)(use & 1));
      if (!__all_sync(0xffffffffu, ok)) {
        fail = true;
        break;
      }
      const int fl = s_fl[slot], nJ = s_nJ[slot], T = s_T[slot], v0 = s_v0[slot];
      const int4 e4[2] = {*reinterpret_cast<const int4*>(&s_ev[slot][vv0]),
                          *reinterpret_cast<const int4*>(&s_ev[slot][vv0 + 4])};
      __syncwarp();
      if (fl & XF_END) break;
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar_free[slot])) : "memory");
      if (T != lastT) {
        g = tile_point(G, T, p);
        lastT = T;
      }
      const int vbase = v0 + vv0;  // this warp's first vector of the chunk
      double* o = out + (size_t)vbase * ng + (g >= 0 ? g : 0);
      const bool full = vbase + 8 <= m;
      if (nJ > 0) {
        const int tb = (int)(cgm & 1);
        ok = mbar_wait(smem_addr(&bar_md[tb]), (uint32_t)((cgm >> 1) & 1));
        if (!__all_sync(0xffffffffu, ok)) {
          fail = true;
          break;
        }
        ++cgm;
        tc_fence_after();
        const uint32_t la = lane_q + (uint32_t)(tb * XT_COLS);
        const int ev[8] = {e4[0].x, e4[0].y, e4[0].z, e4[0].w, e4[1].x, e4[1].y, e4[1].z, e4[1].w};
        const bool wide = nJ > XKS;
        // four vectors at a time: six diagonal sums each
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t f[DIG][4];
#pragma unroll
          for (int d = 0; d < DIG; ++d) tmem_ld4(la + (uint32_t)(d * XN + 4 * hh), f[d]);
          tmem_wait_ld();
          if (hh == 1) {  // the buffer is read: the next MMAs may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar_tf[tb])) : "memory");
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // sum_d D_d 256^(5 - d) in three 32-bit pairs; |D_d| < 2^22 except
            // D_4 and D_5 of lists longer than 16 (below 2^23): those by the
            // conversion instruction
            const int t01 = small_float_int(f[0][u]) * 256 + small_float_int(f[1][u]);
            const int t23 = small_float_int(f[2][u]) * 256 + small_float_int(f[3][u]);
            const int d4 = wide ? __float2int_rz(__uint_as_float(f[4][u])) : small_float_int(f[4][u]);
            const int d5 = wide ? __float2int_rz(__uint_as_float(f[5][u])) : small_float_int(f[5][u]);
            const int t45 = d4 * 256 + d5;
            const long long base = ((long long)t01 << 32) + (long long)t45;
            const long long acc = base + (long long)t23 * 65536LL;
            const double val = scaled_i64_rz_cvt(acc, ev[4 * hh + u] - 1022 - 55);
            if (g >= 0 && (full || vbase + 4 * hh + u < m)) o[(size_t)(4 * hh + u) * ng] = val;
          }
        }
      } else if (g >= 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (full || vbase + u < m) o[(size_t)u * ng] = 0.0;
      }
    }
    if (fail && lane == 0) s_fail = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && s_fail) atomicOr(status, SEA_FLAG_WAIT);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

}  // namespace


size_t w_digits_bytes(long long slots) {
  return (size_t)std::max(slots, 1LL) * 2 * DIG * 8 * sizeof(uint4) +
         (size_t)std::max(slots, 1LL) * 2 * sizeof(int);
}

cudaError_t launch_w_digits(cudaStream_t st, const double* W, const TileGeom& G, size_t ng,
                            int n_tiles, int max_list, const int* tptr, const int* tlist,
                            long long slots, void* wbuf) {
  if (n_tiles <= 0 || max_list <= 0) return cudaSuccess;
  uint4* wdig = (uint4*)wbuf;
  int* wexp = (int*)(wdig + (size_t)std::max(slots, 1LL) * 2 * DIG * 8);
  const int ngroups = (max_list + 7) / 8;
  const long long warps = (long long)n_tiles * 2 * ngroups;
  k_w_digits<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(W, G, ng, n_tiles, ngroups, tptr, tlist,
                                                          wdig, wexp);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, looked up once through the
// runtime (no link-time dependence on the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// The 4D view (x, y, z, row) of A for the tensor-memory-accelerator path;
// false where it does not apply (odd nx: rows not 16-byte strided; A not
// 16-byte aligned; no driver entry point).
static bool make_a_map(const double* A, int m, const TileGeom& G, CUtensorMap* map) {
  if ((G.nx & 1) || (((uintptr_t)A) & 15)) return false;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dim[4] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz, (cuuint64_t)m};
  const cuuint64_t stride[3] = {(cuuint64_t)G.nx * 8, (cuuint64_t)G.nx * G.ny * 8,
                                (cuuint64_t)G.nx * G.ny * G.nz * 8};
  const cuuint32_t box[4] = {TX, TY, 1, MBLK};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)A, dim, stride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t wx_digits_bytes(int n_tiles, long long slots) {
  return (size_t)std::max(n_tiles, 1) * XA_TILE + (size_t)std::max(slots, 1LL) * sizeof(int);
}

cudaError_t launch_wx_digits(cudaStream_t st, const double* W, const TileGeom& G, size_t ng,
                             int n_tiles, const int* tptr, const int* tlist, const int* tsub,
                             void* wxbuf) {
  if (n_tiles <= 0) return cudaSuccess;
  uint4* wx = (uint4*)wxbuf;
  int* wxexp = (int*)((unsigned char*)wxbuf + (size_t)n_tiles * XA_TILE);
  k_wx_digits<<<n_tiles, MBLK, 0, st>>>(W, G, ng, n_tiles, tptr, tlist, tsub, wx, wxexp);
  return cudaGetLastError();
}

cudaError_t launch_expand_tc(cudaStream_t st, int device, const void* wxbuf, const TileGeom& G,
                             size_t ng, int n_tiles, const int* tptr, const int* tlist,
                             const double* H, long long hj, long long hv, int m, bool negate,
                             double* out, int* evbuf, int* queue, unsigned* status) {
  static bool attr_set[64] = {};
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[device]) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_expand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XE_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[device] = true;
  }
  if (n_tiles <= 0 || m <= 0) return cudaSuccess;
  const uint4* wx = (const uint4*)wxbuf;
  const int* wxexp = (const int*)((const unsigned char*)wxbuf + (size_t)n_tiles * XA_TILE);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_expand_ev<<<dim3((m + 127) / 128, n_tiles), 128, 0, st>>>(tptr, tlist, wxexp, H, hj, hv, m,
                                                             evbuf);
  k_expand_tc<<<std::min(nsm, n_tiles), XE_THREADS, XE_SMEM, st>>>(
      wx, wxexp, G, ng, n_tiles, tptr, tlist, H, hj, hv, m, negate ? 1 : 0, out, evbuf, queue,
      status);
  return cudaGetLastError();
}

int expand_tc_max_list() { return XJ; }

cudaError_t launch_gram_tc(cudaStream_t st, int device, const double* A, int m, const TileGeom& G,
                           size_t ng, int n_tiles, const int* tptr, long long slots,
                           const void* wbuf, double* partial, int* queue, unsigned* status) {
  static bool attr_set[64] = {};
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[device]) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc_ldg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GT_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GT2_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[device] = true;
  }
  const uint4* wdig = (const uint4*)wbuf;
  const int* wexp = (const int*)(wdig + (size_t)std::max(slots, 1LL) * 2 * DIG * 8);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int grid = std::min(nsm, std::max(n_tiles, 1));
  alignas(64) CUtensorMap map;
  if (make_a_map(A, m, G, &map))
    k_gram_tc<<<grid, GT2_THREADS, GT2_SMEM, st>>>(map, m, G, n_tiles, tptr, wdig, wexp, partial,
                                                  queue, status);
  else
    k_gram_tc_ldg<<<grid, GT_THREADS, GT_SMEM, st>>>(A, m, G, ng, n_tiles, tptr, wdig, wexp,
                                                     partial, queue, status);
  return cudaGetLastError();
}

}  // namespace sea
