// chol_flow.cu -- the mixed form's Cholesky of -Mbar, L^-1 and E_xx^ACE in
// one launch (Sec. II C, Eq. Vace; Eq. exx_ace):
//
//   -Mbar = L L^T,  Mbar = (M + M^T) / 2;   Linv = L^-1;
//   E_xx^ACE = -sum_ik <phi_i|xi_k>^2 = -|| L^-1 M^T ||_F^2      (xi = W L^-T)
//
// The n x n matrices are cut into 32 x 32 blocks, nb = ceil(n / 32) per
// side (the last block padded with the identity in A = -Mbar and zeros in
// M).  The work is a set of block tasks, one CTA each; a task waits for the
// tasks whose blocks it reads through one flag per task in global memory
// and publishes its own block by setting its flag.  For block column s:
//   D_s    S = A_ss - sum_{k<s} L_sk L_sk^T,  L_ss = chol(S)  (1/L_ss(c,c) kept)
//   Y_s    Linv_ss = L_ss^-1                                    (L_ss Y = I)
//   P_is   i > s:  S = A_is - sum_{k<s} L_ik L_sk^T,  L_is = S L_ss^-T
//   X_sj   j < s:  Linv_sj = -L_ss^-1 sum_{k=j}^{s-1} L_sk Linv_kj
//   Z_sq   all q:  Z_sq = L_ss^-1 ((M^T)_sq - sum_{k<s} L_sk Z_kq),
//                  E_sq = sum of the squares of Z_sq        (Z = L^-1 M^T)
// and a last task F adds the E_sq in a fixed order.  The sums over k are
// taken as their inputs appear, so each step s adds to the chain one block
// product, one 32 x 32 factorization and one triangular solve.
//
// Tasks are numbered step by step in the order above; every task reads only
// lower-numbered ones.  CTA b takes tasks b, b + G, b + 2G, ... in turn, so
// the lowest unfinished task always has its inputs; the launch is
// cooperative (all G CTAs resident), hence it cannot deadlock.  Every flag
// wait is bounded: on expiry the task sets SEA_FLAG_WAIT and goes on, so
// the launch always ends.
//
// Arithmetic: double-float (hi + lo FP32 pairs, about 48 bits) on the FP32
// pipes throughout -- on this part a warp's FP64 instruction holds the FP64
// unit of its SM sub-partition for about 64 cycles, which would make the
// one-SM block steps of the chain slow.  Inputs (M) and outputs (L, Linv,
// E_xx^ACE) are FP64.  Every sum is taken in a fixed order, so repeated
// launches give the same bits.
#include <cuda_runtime.h>

#include <algorithm>

#include "sea_internal.cuh"

namespace sea {
namespace {

constexpr int FB = 32;   // block side
constexpr int FT = 256;  // threads per CTA
constexpr long long FLOW_WAIT_CYCLES = 2000000000LL;

struct FlowArgs {
  const double* M;  // n x n, row-major
  int n, nb;
  double* L;      // out: n x n, zeros above the diagonal
  double* Linv;   // out: n x n, zeros above the diagonal
  float2* Lb;     // DF blocks of L, block (i, j) at (i nb + j) * 1024
  float2* Rb;     // DF 1 / L(c, c), 32 per diagonal block
  float2* Xb;     // DF blocks of L^-1
  float2* Zb;     // DF blocks of Z = L^-1 M^T
  float2* Eb;     // DF sums of squares of the Z blocks
  int* flag;      // one per task, zero before the launch
  unsigned* status;
  double* exx;    // out: E_xx^ACE
};

struct SBlk {
  float h[FB][FB + 1];
  float l[FB][FB + 1];
};

__device__ __forceinline__ DF sget(const SBlk& b, int r, int c) { return DF{b.h[r][c], b.l[r][c]}; }
__device__ __forceinline__ void sput(SBlk& b, int r, int c, DF v) {
  b.h[r][c] = v.hi;
  b.l[r][c] = v.lo;
}
__device__ __forceinline__ DF shfl_df(DF v, int src) {
  return DF{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ DF df_of(double x) {
  const float2 s = split64(x);
  return DF{s.x, s.y};
}

// task numbering: step s holds 2 nb + 1 tasks
struct Tasks {
  int nb;
  __device__ int per() const { return 2 * nb + 1; }
  __device__ int D(int s) const { return s * per(); }
  __device__ int Y(int s) const { return D(s) + 1; }
  __device__ int P(int i, int s) const { return D(s) + 1 + (i - s); }
  __device__ int X(int s, int j) const { return D(s) + 1 + (nb - s) + j; }
  __device__ int Z(int s, int q) const { return D(s) + nb + 1 + q; }
  __device__ int F() const { return nb * per(); }
};

// Thread 0 waits until task t has published; then the CTA may read it.
__device__ void wait_task(const FlowArgs& A, int t) {
  if (threadIdx.x == 0) {
    const int* f = A.flag + t;
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v == 0) {
      const long long t0 = clock64();
      for (;;) {
        __nanosleep(64);
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v != 0) break;
        if (clock64() - t0 > FLOW_WAIT_CYCLES) {
          atomicOr(A.status, SEA_FLAG_WAIT);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// After a barrier (the CTA's stores precede it), thread 0 fences and sets
// the flag of task t with a release store; a reader's acquire load of the
// flag followed by its own barrier then orders its CTA's reads after them.
__device__ void publish(const FlowArgs& A, int t) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int* f = A.flag + t;
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(1) : "memory");
  }
}

// DF block from global (L2: written by other CTAs during this launch) into
// shared memory, transposed if tr.
__device__ void load_blk(SBlk& b, const float2* src, bool tr) {
  for (int e = threadIdx.x; e < FB * FB; e += FT) {
    const float2 v = __ldcg(src + e);
    const int r = e >> 5, c = e & 31;
    if (tr) {
      b.h[c][r] = v.x;
      b.l[c][r] = v.y;
    } else {
      b.h[r][c] = v.x;
      b.l[r][c] = v.y;
    }
  }
}

// This thread's four elements (r, c) of a block: r = ty + 16 (e >> 1),
// c = tx + 16 (e & 1).
__device__ __forceinline__ int er(int e) { return (threadIdx.x >> 4) + 16 * (e >> 1); }
__device__ __forceinline__ int ec(int e) { return (threadIdx.x & 15) + 16 * (e & 1); }

// acc(r, c) += sign sum_m a(r, m) b(c, m), m ascending.  Loops stay rolled
// here and below: each CTA runs its task's code once, from a cold
// instruction cache, so the code's size costs more than its loop overhead.
__device__ void acc_prod(DF acc[4], const SBlk& a, const SBlk& b, float sign) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll 1
  for (int m = 0; m < FB; ++m) {
    const DF a0 = DF{sign * a.h[ty][m], sign * a.l[ty][m]};
    const DF a1 = DF{sign * a.h[ty + 16][m], sign * a.l[ty + 16][m]};
    const DF b0 = sget(b, tx, m), b1 = sget(b, tx + 16, m);
    acc[0] = df_fma(a0, b0, acc[0]);
    acc[1] = df_fma(a0, b1, acc[1]);
    acc[2] = df_fma(a1, b0, acc[2]);
    acc[3] = df_fma(a1, b1, acc[3]);
  }
}

// A = -(M + M^T) / 2 at global (I, J), the identity beyond n.
__device__ __forceinline__ DF a_elem(const FlowArgs& A, int I, int J) {
  if (I >= A.n || J >= A.n) return DF{I == J ? 1.f : 0.f, 0.f};
  const DF s = df_add(df_of(A.M[(size_t)I * A.n + J]), df_of(A.M[(size_t)J * A.n + I]));
  return DF{-0.5f * s.hi, -0.5f * s.lo};
}

// L_ss and its reciprocal pivots into sL (scaled: sL(c, m) = L(c, m) / L(m, m)
// for m < c, the form the solves use) and rinv.
__device__ void load_diag_scaled(const FlowArgs& A, int s, SBlk& sL, DF* rinv) {
  if (threadIdx.x < FB) {
    const float2 v = __ldcg(A.Rb + s * FB + threadIdx.x);
    rinv[threadIdx.x] = DF{v.x, v.y};
  }
  __syncthreads();
  const float2* src = A.Lb + ((size_t)s * A.nb + s) * FB * FB;
  for (int e = threadIdx.x; e < FB * FB; e += FT) {
    const int r = e >> 5, c = e & 31;
    const float2 v = __ldcg(src + e);
    const DF x = (c < r) ? df_mul(DF{v.x, v.y}, rinv[c]) : DF{0.f, 0.f};
    sput(sL, r, c, x);
  }
  __syncthreads();
}

// Forward substitution for every row rho of R: x with L x = R(rho, :)^T,
// written back to R(rho, :).  sL holds L scaled as in load_diag_scaled:
// with a_c = x_c L(c, c), step m takes a_m (final) and subtracts
// (L(c, m) / L(m, m)) a_m from a_c for c > m; at the end x_c = a_c / L(c, c).
// Warp w takes rows w, w + 8, w + 16, w + 24; lane = c.
__device__ void solve_rows(SBlk& R, const SBlk& sL, const DF* rinv) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DF x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = sget(R, w + 8 * q, lane);
#pragma unroll 2
  for (int m = 0; m < FB - 1; ++m) {
    const DF nl = df_neg(sget(sL, lane, m));
    const bool upd = lane > m;
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // selects, not branches: the four chains stay interleaved
      const DF y = df_fma(nl, shfl_df(x[q], m), x[q]);
      x[q] = upd ? y : x[q];
    }
  }
  const DF ri = rinv[lane];
#pragma unroll
  for (int q = 0; q < 4; ++q) sput(R, w + 8 * q, lane, df_mul(x[q], ri));
  __syncthreads();
}

// 1 / sqrt(d) for d > 0 in double-float, on the pivot chain: the FP32
// reciprocal square root, one Newton step in FP32 (relative error about
// 2^-23), one in double-float (about 2^-46): r + r (1 - d r^2) / 2 with
// d r^2 formed from the exact square of r.
__device__ __forceinline__ DF pivot_rsqrt(DF d) {
  float r = rsqrtf(d.hi);
  r = r * fmaf(-0.5f * d.hi, r * r, 1.5f);
  const float q = r * r;
  const float qe = fmaf(r, r, -q);  // r^2 = q + qe exactly
  const DF t = df_mul(d, DF{q, qe});
  const float e = (1.0f - t.hi) - t.lo;
  return df_fast_two_sum(r, (0.5f * r) * e);
}

// Cholesky of the 32 x 32 block in sS by the CTA's 8 warps: warp w holds
// the columns 4w .. 4w + 3 (lane = row).  In turn, warp b takes the pivots
// of its four columns (each column then updates the warp's later columns
// through shuffles, with no barrier), writes them to sL and, after a
// barrier, every later warp subtracts their rank-4 product from its columns.
// The pivot chain thus leaves the warp once per four columns.  1 / L(k, k)
// goes to rinv.  Returns false on a non-positive pivot (its column is then 0).
__device__ bool factor_block(const SBlk& sS, SBlk& sL, DF* rinv) {
  __shared__ int bad;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DF a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = sget(sS, lane, 4 * w + q);
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
#pragma unroll 1
  for (int b = 0; b < FB / 4; ++b) {
    if (w == b) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * b + q;
        const DF d = shfl_df(a[q], k);
        const bool pos = d.hi > 0.f;
        const DF r = pivot_rsqrt(pos ? d : DF{1.f, 0.f});
        const DF rr = pos ? r : DF{0.f, 0.f};
        const DF l = df_mul(lane == k ? d : a[q], rr);
        a[q] = lane >= k ? l : DF{0.f, 0.f};
        if (lane == k) {
          rinv[k] = rr;
          if (!pos) bad = 1;
        }
        const DF nl = df_neg(a[q]);
#pragma unroll
        for (int q2 = q + 1; q2 < 4; ++q2) a[q2] = df_fma(nl, shfl_df(a[q], 4 * b + q2), a[q2]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) sput(sL, lane, 4 * b + q, a[q]);
    }
    __syncthreads();
    if (w > b) {
      DF li[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) li[q] = df_neg(sget(sL, lane, 4 * b + q));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 4 * w + q;
        const DF t = df_dot2(li[0], sget(sL, c, 4 * b), li[1], sget(sL, c, 4 * b + 1));
        const DF u = df_dot2(li[2], sget(sL, c, 4 * b + 2), li[3], sget(sL, c, 4 * b + 3));
        a[q] = df_add(a[q], df_add(t, u));
      }
    }
  }
  __syncthreads();
  return bad == 0;
}

// Block (bi, bj) of an FP64 n x n output from R (rows r, columns c), or
// zeros; only indices below n.
__device__ void store_f64(const FlowArgs& A, double* out, int bi, int bj, const SBlk* R, bool lower_only) {
  for (int e = threadIdx.x; e < FB * FB; e += FT) {
    const int r = e >> 5, c = e & 31;
    const int I = bi * FB + r, J = bj * FB + c;
    if (I >= A.n || J >= A.n) continue;
    double v = 0.0;
    if (R && (!lower_only || c <= r)) v = df_to_double(sget(*R, r, c));
    out[(size_t)I * A.n + J] = v;
  }
}

__device__ void store_df(float2* dst, const SBlk& R, bool tr) {
  for (int e = threadIdx.x; e < FB * FB; e += FT) {
    const int r = e >> 5, c = e & 31;
    const DF v = tr ? sget(R, c, r) : sget(R, r, c);
    dst[e] = make_float2(v.hi, v.lo);
  }
}

__global__ void __launch_bounds__(FT) k_chol_flow(FlowArgs A) {
  __shared__ SBlk sA, sB, sL, sR;
  __shared__ DF rinv[FB];
  const Tasks T{A.nb};
  const int nb = A.nb, per = T.per();
  const int ntask = T.F() + 1;
  for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
    DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (t == T.F()) {
      // F: E_xx^ACE = -sum_{s, q} E_sq, s then q ascending
      for (int u = 0; u < nb * nb; ++u) wait_task(A, T.Z(u / nb, u % nb));
      if (threadIdx.x < 32) {
        DF sum{0.f, 0.f};
        for (int u = threadIdx.x; u < nb * nb; u += 32) {
          const float2 v = __ldcg(A.Eb + u);
          sum = df_add(sum, DF{v.x, v.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum = df_add(sum, shfl_df(sum, (threadIdx.x + o) & 31));
        if (threadIdx.x == 0) *A.exx = -df_to_double(sum);
      }
      continue;
    }
    const int s = t / per, r = t % per;
    if (r == 0) {
      // D_s
      for (int e = 0; e < 4; ++e) acc[e] = a_elem(A, s * FB + er(e), s * FB + ec(e));
      for (int k = 0; k < s; ++k) {
        wait_task(A, T.P(s, k));
        const float2* lk = A.Lb + ((size_t)s * nb + k) * FB * FB;
        load_blk(sA, lk, false);
        __syncthreads();
        acc_prod(acc, sA, sA, -1.f);
        __syncthreads();
      }
      for (int e = 0; e < 4; ++e) sput(sR, er(e), ec(e), acc[e]);
      __syncthreads();
      if (!factor_block(sR, sL, rinv) && threadIdx.x == 0) atomicOr(A.status, SEA_FLAG_NOT_PD);
      store_df(A.Lb + ((size_t)s * nb + s) * FB * FB, sL, false);
      if (threadIdx.x < FB) A.Rb[s * FB + threadIdx.x] = make_float2(rinv[threadIdx.x].hi, rinv[threadIdx.x].lo);
      publish(A, t);  // the FP64 outputs after the hand-over: only the caller reads them
      store_f64(A, A.L, s, s, &sL, true);
    } else if (r == 1) {
      // Y_s: L_ss Y = I, by rows of Y^T
      wait_task(A, T.D(s));
      load_diag_scaled(A, s, sL, rinv);
      for (int e = threadIdx.x; e < FB * FB; e += FT) sput(sR, e >> 5, e & 31, DF{(e >> 5) == (e & 31) ? 1.f : 0.f, 0.f});
      __syncthreads();
      solve_rows(sR, sL, rinv);  // sR = Y^T
      store_df(A.Xb + ((size_t)s * nb + s) * FB * FB, sR, true);
      publish(A, t);
      for (int e = threadIdx.x; e < FB * FB; e += FT) {
        const int rr = e >> 5, c = e & 31;
        const int I = s * FB + rr, J = s * FB + c;
        if (I < A.n && J < A.n) A.Linv[(size_t)I * A.n + J] = c <= rr ? df_to_double(sget(sR, c, rr)) : 0.0;
      }
    } else if (r <= nb - s) {
      // P_is
      const int i = s + r - 1;
      for (int e = 0; e < 4; ++e) acc[e] = a_elem(A, i * FB + er(e), s * FB + ec(e));
      for (int k = 0; k < s; ++k) {
        wait_task(A, T.P(i, k));
        wait_task(A, T.P(s, k));
        load_blk(sA, A.Lb + ((size_t)i * nb + k) * FB * FB, false);
        load_blk(sB, A.Lb + ((size_t)s * nb + k) * FB * FB, false);
        __syncthreads();
        acc_prod(acc, sA, sB, -1.f);
        __syncthreads();
      }
      wait_task(A, T.D(s));
      load_diag_scaled(A, s, sL, rinv);
      for (int e = 0; e < 4; ++e) sput(sR, er(e), ec(e), acc[e]);
      __syncthreads();
      solve_rows(sR, sL, rinv);  // rows of L_is
      store_df(A.Lb + ((size_t)i * nb + s) * FB * FB, sR, false);
      publish(A, t);
      store_f64(A, A.L, i, s, &sR, false);
      store_f64(A, A.L, s, i, nullptr, false);
    } else if (r <= nb) {
      // X_sj
      const int j = r - (nb - s + 1);
      for (int k = j; k < s; ++k) {
        wait_task(A, T.P(s, k));
        wait_task(A, k == j ? T.Y(j) : T.X(k, j));
        load_blk(sA, A.Lb + ((size_t)s * nb + k) * FB * FB, false);
        load_blk(sB, A.Xb + ((size_t)k * nb + j) * FB * FB, true);
        __syncthreads();
        acc_prod(acc, sA, sB, 1.f);
        __syncthreads();
      }
      wait_task(A, T.D(s));
      load_diag_scaled(A, s, sL, rinv);
      for (int e = 0; e < 4; ++e) sput(sR, ec(e), er(e), df_neg(acc[e]));  // (-T)^T
      __syncthreads();
      solve_rows(sR, sL, rinv);  // X_sj^T
      store_df(A.Xb + ((size_t)s * nb + j) * FB * FB, sR, true);
      publish(A, t);
      for (int e = threadIdx.x; e < FB * FB; e += FT) {
        const int rr = e >> 5, c = e & 31;
        const int I = s * FB + rr, J = j * FB + c;
        if (I < A.n && J < A.n) {
          A.Linv[(size_t)I * A.n + J] = df_to_double(sget(sR, c, rr));
          A.Linv[(size_t)J * A.n + I] = 0.0;
        }
      }
    } else {
      // Z_sq and E_sq
      const int q = r - nb - 1;
      for (int e = 0; e < 4; ++e) {
        const int I = q * FB + ec(e), J = s * FB + er(e);  // (M^T)(s-row, q-col) = M(q-row, s-col)
        acc[e] = (I < A.n && J < A.n) ? df_of(A.M[(size_t)I * A.n + J]) : DF{0.f, 0.f};
      }
      for (int k = 0; k < s; ++k) {
        wait_task(A, T.P(s, k));
        wait_task(A, T.Z(k, q));
        load_blk(sA, A.Lb + ((size_t)s * nb + k) * FB * FB, false);
        load_blk(sB, A.Zb + ((size_t)k * nb + q) * FB * FB, true);
        __syncthreads();
        acc_prod(acc, sA, sB, -1.f);
        __syncthreads();
      }
      wait_task(A, T.D(s));
      load_diag_scaled(A, s, sL, rinv);
      for (int e = 0; e < 4; ++e) sput(sR, ec(e), er(e), acc[e]);
      __syncthreads();
      solve_rows(sR, sL, rinv);  // Z_sq^T
      store_df(A.Zb + ((size_t)s * nb + q) * FB * FB, sR, true);
      // E_sq: the squares in a fixed order (thread partials, then a tree)
      __shared__ DF red[FT / 32];
      DF e2{0.f, 0.f};
      for (int e = threadIdx.x; e < FB * FB; e += FT) {
        const DF v = sget(sR, e & 31, e >> 5);
        e2 = df_fma(v, v, e2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const DF u = shfl_df(e2, (threadIdx.x + o) & 31);
        e2 = df_add(e2, u);
      }
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
      __syncthreads();
      if (threadIdx.x == 0) {
        DF sum = red[0];
        for (int w = 1; w < FT / 32; ++w) sum = df_add(sum, red[w]);
        A.Eb[s * nb + q] = make_float2(sum.hi, sum.lo);
      }
      publish(A, t);
    }
    __syncthreads();
  }
}

}  // namespace

// DF scratch of the launch (bytes) for n orbitals.
size_t chol_flow_bytes(int n) {
  const size_t nb = (size_t)(n + FB - 1) / FB;
  const size_t ntask = nb * (2 * nb + 1) + 1;
  return (3 * nb * nb * FB * FB + nb * FB + nb * nb) * sizeof(float2) + ntask * sizeof(int) + 256;
}

// Enqueues the flag reset and the cooperative launch on stream st.
cudaError_t launch_chol_flow(cudaStream_t st, int device, const double* M, int n, double* L,
                             double* Linv, void* scratch, unsigned* status, double* exx) {
  int occ = 0, nsm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chol_flow, FT, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorLaunchOutOfResources;
  const int nb = (n + FB - 1) / FB;
  const int ntask = nb * (2 * nb + 1) + 1;
  FlowArgs A;
  A.M = M;
  A.n = n;
  A.nb = nb;
  A.L = L;
  A.Linv = Linv;
  float2* p = (float2*)scratch;
  const size_t blk = (size_t)nb * nb * FB * FB;
  A.Lb = p;
  A.Xb = p + blk;
  A.Zb = p + 2 * blk;
  A.Rb = p + 3 * blk;
  A.Eb = A.Rb + (size_t)nb * FB;
  A.flag = (int*)(A.Eb + (size_t)nb * nb);
  A.status = status;
  A.exx = exx;
  e = cudaMemsetAsync(A.flag, 0, (size_t)ntask * sizeof(int), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min(ntask, occ * nsm));
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_chol_flow, A);
}

}  // namespace sea
