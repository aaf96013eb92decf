// sea_internal.cuh -- device helpers and the context of the GB300 exx engine.
//
// Everything here belongs to the CUDA library (libsea.so).  It is written
// from the paper's equations; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "../../include/sea.h"

#define SEA_LMAX 6
#define SEA_NQ ((SEA_LMAX + 1) * (SEA_LMAX + 1))
// monomials x^a y^b z^c with a + b + c <= SEA_LMAX
#define SEA_NMONO ((SEA_LMAX + 1) * (SEA_LMAX + 2) * (SEA_LMAX + 3) / 6)
// per pair: the moments Qs (SEA_NQ), then the multipole potential's
// coefficients in the Kelvin-inverted variables (SEA_NMONO)
#define SEA_QSTRIDE (SEA_NQ + SEA_NMONO)
#define SEA_FDP 6  // stencil half width: O(h^12) second difference (App. C)

// Status bits written by kernels (device word, read back by the host).
#define SEA_FLAG_CG_CAP 1u
#define SEA_FLAG_NOT_PD 2u
#define SEA_FLAG_BOUNDS 4u
#define SEA_FLAG_NONFINITE 8u
#define SEA_FLAG_WAIT 16u  // a bounded wait on a tensor-core completion expired
#define SEA_FLAG_TIMEOUT 32u  // the CG's time budget (sea_params.timeout_ms) was spent
#define SEA_FLAG_NORM 64u     // an orbital's norm is off 1 by more than orth_tol

// Slot (in doubles) of E_xx^ACE in the context's exx_dev buffer (the first
// five hold sea_apply_vxx's E_xx and CG statistics).
#define SEA_EXX_ACE_SLOT 6

// At most this many chunks per pipelined host-buffer call.
#define SEA_XCHUNKS_MAX 64

namespace sea {

// NVTX ranges of an entry point and its stages, for timeline tools (Nsight
// Systems, or ncu's --nvtx filters); without an attached tool each push and
// pop is a test of one function pointer.  The ranges mark where the host
// enqueues each stage's launches; the stage times on the device are the
// CUDA-event times in sea_stats.  stage() closes the previous stage's range
// and opens the next; the destructor closes the open stage and the call.
struct Trace {
  explicit Trace(const char* call) { nvtxRangePushA(call); }
  void stage(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~Trace() {
    if (open) nvtxRangePop();
    nvtxRangePop();
  }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
  bool open = false;
};

__host__ __device__ inline int wrapi(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

__host__ __device__ inline int lmi(int l, int m) { return l * l + l + m; }

// Position of x^a y^b z^c among the SEA_NMONO monomials (a-major, then b,
// then c), the layout of the potential's coefficients.
__host__ __device__ constexpr int mono_k(int a, int b, int c) {
  int k = 0;
  for (int i = 0; i < a; ++i) k += (SEA_LMAX - i + 1) * (SEA_LMAX - i + 2) / 2;
  for (int j = 0; j < b; ++j) k += SEA_LMAX - a - j + 1;
  return k + c;
}

// Real solid harmonics in a rescaled basis D_lm = C_lm / kappa_lm, where
// C_lm are the Racah-normalized real regular solid harmonics
// (C_l0 = r^l P_l(cos theta)).  The scaling is chosen so that the
// recurrences carry no per-term normalization:
//   D_00 = 1, D_11 = x, D_1-1 = y,
//   D_{l+1,l+1} = x D_ll - y D_l,-l,   D_{l+1,-(l+1)} = y D_ll + x D_l,-l,
//   D_{l+1,m} = z D_lm - gam_lm r^2 D_{l-1,m}   (|m| <= l; no second term
//                                                 when |m| = l).
// With Q_lm = sum rho C_lm dV the multipole potential of Eq. me is
//   v(r) = sum_lm Q_lm C_lm(r) / r^(2l+1)
// (the orthonormal form 4 pi Q Y / ((2l+1) r^(l+1)), the (2l+1)/(4 pi)
// normalization folded into C).  Kelvin inversion, u = r / r^2, gives
// C_lm(r) / r^(2l+1) = C_lm(u) / r, so
//   v(r) = (1/r) sum_lm Qs_lm D_lm(u),   Qs_lm = kappa_lm^2 sum rho D_lm dV,
// the D_lm(u) from the same recurrence with r^2 replaced by |u|^2 = 1/r^2.
struct HarmCoef {
  double gam[SEA_LMAX][2 * SEA_LMAX + 1];
  double kap2[SEA_NQ];
  // D_lm as a homogeneous polynomial of degree l:
  //   D_lm(x, y, z) = sum_{a + b <= l} cart[lm][a][b] x^a y^b z^(l - a - b)
  // (the recurrence above carried out on coefficient arrays)
  double cart[SEA_NQ][SEA_LMAX + 1][SEA_LMAX + 1];
  float gam_hi[SEA_LMAX][2 * SEA_LMAX + 1];  // gam = gam_hi + gam_lo (double-float)
  float gam_lo[SEA_LMAX][2 * SEA_LMAX + 1];
};
// Each translation unit that evaluates harmonics holds its own copy (the
// library is built without relocatable device code) and uploads it through
// its own upload_harmonics_<unit>() at context creation.
static __constant__ HarmCoef c_harm;

HarmCoef make_harmonic_coefficients();
static inline cudaError_t upload_harmonics_here() {
  const HarmCoef h = make_harmonic_coefficients();
  return cudaMemcpyToSymbol(c_harm, &h, sizeof(h));
}

// acc[lm] += w * D_lm(x, y, z) (regular, rescaled basis), level by level.
__device__ __forceinline__ void harm_accumulate(double w, double x, double y, double z,
                                                double* acc) {
  const double r2 = x * x + y * y + z * z;
  double D[SEA_NQ];
  D[0] = 1.0;
  D[lmi(1, 1)] = x;
  D[lmi(1, -1)] = y;
  D[lmi(1, 0)] = z;
  acc[0] += w;
  acc[lmi(1, -1)] = fma(w, y, acc[lmi(1, -1)]);
  acc[lmi(1, 0)] = fma(w, z, acc[lmi(1, 0)]);
  acc[lmi(1, 1)] = fma(w, x, acc[lmi(1, 1)]);
#pragma unroll
  for (int l = 1; l < SEA_LMAX; ++l) {
    D[lmi(l + 1, l + 1)] = fma(x, D[lmi(l, l)], -y * D[lmi(l, -l)]);
    D[lmi(l + 1, -(l + 1))] = fma(y, D[lmi(l, l)], x * D[lmi(l, -l)]);
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      if (m >= -(l - 1) && m <= l - 1)
        D[lmi(l + 1, m)] = fma(z, D[lmi(l, m)], -(c_harm.gam[l][m + SEA_LMAX] * r2) * D[lmi(l - 1, m)]);
      else
        D[lmi(l + 1, m)] = z * D[lmi(l, m)];
    }
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m) acc[lmi(l + 1, m)] = fma(w, D[lmi(l + 1, m)], acc[lmi(l + 1, m)]);
  }
}

// Multipole potential at r = (x, y, z) != 0 (relative to the expansion
// centre) from the rescaled moments Qs (shared or global memory, zero beyond
// the requested l_max): v = (1/r) sum Qs_lm D_lm(r / r^2).
__device__ __forceinline__ double me_potential(const double* __restrict__ Q, double x,
                                               double y, double z) {
  const double ir2 = 1.0 / (x * x + y * y + z * z);
  const double ux = x * ir2, uy = y * ir2, uz = z * ir2;
  double D[SEA_NQ];
  D[0] = 1.0;
  D[lmi(1, 1)] = ux;
  D[lmi(1, -1)] = uy;
  D[lmi(1, 0)] = uz;
  double v = Q[0];
  v = fma(Q[lmi(1, -1)], uy, v);
  v = fma(Q[lmi(1, 0)], uz, v);
  v = fma(Q[lmi(1, 1)], ux, v);
#pragma unroll
  for (int l = 1; l < SEA_LMAX; ++l) {
    D[lmi(l + 1, l + 1)] = fma(ux, D[lmi(l, l)], -uy * D[lmi(l, -l)]);
    D[lmi(l + 1, -(l + 1))] = fma(uy, D[lmi(l, l)], ux * D[lmi(l, -l)]);
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      if (m >= -(l - 1) && m <= l - 1)
        D[lmi(l + 1, m)] = fma(uz, D[lmi(l, m)], -(c_harm.gam[l][m + SEA_LMAX] * ir2) * D[lmi(l - 1, m)]);
      else
        D[lmi(l + 1, m)] = uz * D[lmi(l, m)];
    }
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m) v = fma(Q[lmi(l + 1, m)], D[lmi(l + 1, m)], v);
  }
  return v * sqrt(ir2);
}

// v 2^e2 rounded to the nearest FP64 value (ties to even); 0 if below the
// normal range.  Integer operations only.
__device__ __forceinline__ double scaled_i64(long long v, int e2) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
  unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mnt = a >> 11;
  const unsigned rem = (unsigned)(a & 0x7FF);
  if (rem > 0x400u || (rem == 0x400u && (mnt & 1ULL))) ++mnt;
  int ex = 63 - lz + e2 + 1023;
  if (mnt >> 53) {
    mnt >>= 1;
    ++ex;
  }
  if (ex <= 0) return 0.0;
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)ex << 52) | (mnt & 0xFFFFFFFFFFFFFULL)));
}

// v 2^e2 truncated toward zero to FP64 (error below one unit in the last
// place); 0 if below the normal range.  The normalisation works on the two
// 32-bit halves of |v|; integer operations only.
__device__ __forceinline__ double scaled_i64_rz(long long v, int e2) {
  const unsigned long long u = (unsigned long long)v;
  const unsigned sg = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned long long a = v < 0 ? 0ULL - u : u;
  unsigned hi = (unsigned)(a >> 32), lo = (unsigned)a;
  int top = 63;  // bit index of hi's bit 31 in |v|
  if (hi == 0u) {
    hi = lo;
    lo = 0u;
    top = 31;
  }
  if (hi == 0u) return 0.0;
  const int lz = __clz(hi);
  const int ex = top - lz + e2 + 1023;
  if (ex <= 0) return 0.0;
  const unsigned nh = __funnelshift_l(lo, hi, lz), nl = lo << lz;  // leading 1 at bit 63
  const unsigned bh = sg | ((unsigned)ex << 20) | ((nh >> 11) & 0xFFFFFu);
  const unsigned bl = __funnelshift_r(nl, nh, 11);
  return __hiloint2double((int)bh, (int)bl);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2): Knuth's
// two-sum and the fused-multiply-add two-product (Dekker's method), about 48
// significant bits from FP32 operations only.  The mixed form evaluates the
// multipole potential with it: on this part an FP64 instruction of a warp
// costs the issue time of 64 FP32 ones.
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = (a.hi - (s - v)) + (b.hi - v);
  return df_fast_two_sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return df_fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_mul_f(float a, DF b) {  // a exact in FP32
  const float p = a * b.hi;
  const float e = fmaf(a, b.hi, -p);
  return df_fast_two_sum(p, fmaf(a, b.lo, e));
}
// a b + c with one normalisation: the product's high part and c.hi by an
// exact two-sum, every low-order term added to its error, then one fast
// two-sum (15 FP32 operations instead of 17 for df_add(df_mul(a, b), c)).
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
  const float p = a.hi * b.hi;
  const float pe = fmaf(a.hi, b.hi, -p);
  const float s = p + c.hi;
  const float v = s - p;
  const float e = (p - (s - v)) + (c.hi - v);
  return df_fast_two_sum(s, (fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe)) + c.lo) + e);
}
// a b + c d with one normalisation: the two products' high parts by an
// exact two-sum, their errors and cross terms added to its error (19 FP32
// operations instead of 22).  For a b - c d pass df_neg(c).
__device__ __forceinline__ DF df_dot2(DF a, DF b, DF c, DF d) {
  const float p = a.hi * b.hi, q = c.hi * d.hi;
  const float pe = fmaf(a.hi, b.hi, -p), qe = fmaf(c.hi, d.hi, -q);
  const float s = p + q;
  const float v = s - p;
  const float e = (p - (s - v)) + (q - v);
  const float lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe)) + fmaf(c.hi, d.lo, fmaf(c.lo, d.hi, qe));
  return df_fast_two_sum(s, lo + e);
}
// 1 / a: FP32 reciprocal, one Newton step in double-float
__device__ __forceinline__ DF df_rcp(DF a) {
  const float y = 1.0f / a.hi;
  const DF t = df_mul_f(y, a);  // a y = 1 - e
  const float e = (1.0f - t.hi) - t.lo;
  return df_fast_two_sum(y, y * e);
}
// sqrt(a): FP32 square root, one Newton step in double-float
__device__ __forceinline__ DF df_sqrt(DF a) {
  const float s = sqrtf(a.hi);
  const float p = s * s;
  const float pe = fmaf(s, s, -p);
  const float d = ((a.hi - p) - pe) + a.lo;  // a - s^2
  return df_fast_two_sum(s, d * (0.5f / s));
}
// An int |v| < 2^22 as FP32, exactly, without a conversion instruction:
// added to the bit pattern of 1.5 2^23 it lands in the low mantissa bits.
__device__ __forceinline__ float i2f_exact(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
// hi + lo as FP64 with integer operations only: both terms as fixed-point
// integers on the larger one's exponent (bits more than 2^-62 below it
// dropped), one rounding to nearest.  FP32 subnormals count as zero.
__device__ __forceinline__ double df_to_double(DF a) {
  const unsigned bh = __float_as_uint(a.hi), bl = __float_as_uint(a.lo);
  const int eh = (int)((bh >> 23) & 0xFF), el = (int)((bl >> 23) & 0xFF);
  const int E = max(eh, el);
  if (E == 0) return 0.0;
  auto fixed = [&](unsigned b, int e) -> long long {
    if (e == 0) return 0;
    const int sh = E - e;
    if (sh > 62) return 0;
    const long long v = ((long long)((b & 0x7FFFFFu) | 0x800000u) << 38) >> sh;
    return (b >> 31) ? -v : v;
  };
  return scaled_i64(fixed(bh, eh) + fixed(bl, el), E - 150 - 38);
}

// v = hi + lo with integer operations only (no FP64 instruction): hi keeps
// the sign, the exponent and the top 23 mantissa bits (truncation), lo the
// remaining 29 bits, rounded to an FP32 value of the same sign.  |v| below
// the FP32 normal range (2^-126) is flushed to (0, 0).  Relative error of
// hi + lo: <= 2^-47.
__device__ __forceinline__ float2 split64(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e - 1023 + 127 <= 0) return make_float2(0.f, 0.f);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  // lo = (m mod 2^29) 2^(e - 1075) = ((m mod 2^29) 2^-64) 2^(e - 1011); e > 896 keeps
  // the second factor a normal FP32 power of two
  const float l = ((float)(unsigned)(m & 0x1FFFFFFFULL) * 5.421010862427522e-20f) *
                  __uint_as_float((unsigned)(e - 884) << 23);
  return make_float2(hi, __uint_as_float(__float_as_uint(l) | sign));
}

// An FP64 value as a double-float pair, by split64 (no FP64 instruction:
// on this part a warp's FP64 conversion or add holds the FP64 pipe for
// about 64 cycles).
__device__ __forceinline__ DF df_from_double(double x) {
  const float2 s = split64(x);
  return DF{s.x, s.y};
}

// me_potential in double-float: the same recurrences and summation order,
// Q as double-float coefficients.
__device__ __forceinline__ DF me_potential_df(const DF* __restrict__ Q, DF x, DF y, DF z) {
  const DF r2 = df_fma(z, z, df_dot2(x, x, y, y));
  const DF ir2 = df_rcp(r2);
  const DF ux = df_mul(x, ir2), uy = df_mul(y, ir2), uz = df_mul(z, ir2);
  DF Dm[2 * SEA_LMAX + 1], Dc[2 * SEA_LMAX + 1], Dn[2 * SEA_LMAX + 1];  // l-1, l, l+1
#pragma unroll
  for (int k = 0; k < 2 * SEA_LMAX + 1; ++k) Dm[k] = Dc[k] = Dn[k] = DF{0.f, 0.f};
  Dm[SEA_LMAX] = DF{1.f, 0.f};  // l = 0
  Dc[SEA_LMAX + 1] = ux;        // l = 1: m = 1, -1, 0
  Dc[SEA_LMAX - 1] = uy;
  Dc[SEA_LMAX] = uz;
  DF v = Q[0];
  v = df_fma(Q[lmi(1, -1)], uy, v);
  v = df_fma(Q[lmi(1, 0)], uz, v);
  v = df_fma(Q[lmi(1, 1)], ux, v);
#pragma unroll
  for (int l = 1; l < SEA_LMAX; ++l) {
    Dn[SEA_LMAX + l + 1] = df_dot2(ux, Dc[SEA_LMAX + l], df_neg(uy), Dc[SEA_LMAX - l]);
    Dn[SEA_LMAX - l - 1] = df_dot2(uy, Dc[SEA_LMAX + l], ux, Dc[SEA_LMAX - l]);
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      if (m >= -(l - 1) && m <= l - 1) {
        const DF g = df_mul(DF{c_harm.gam_hi[l][m + SEA_LMAX], c_harm.gam_lo[l][m + SEA_LMAX]}, ir2);
        Dn[SEA_LMAX + m] = df_dot2(uz, Dc[SEA_LMAX + m], df_neg(g), Dm[SEA_LMAX + m]);
      } else {
        Dn[SEA_LMAX + m] = df_mul(uz, Dc[SEA_LMAX + m]);
      }
    }
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m) v = df_fma(Q[lmi(l + 1, m)], Dn[SEA_LMAX + m], v);
#pragma unroll
    for (int k = 0; k < 2 * SEA_LMAX + 1; ++k) {
      Dm[k] = Dc[k];
      Dc[k] = Dn[k];
    }
  }
  return df_mul(v, df_sqrt(ir2));
}

// The multipole potential of Eq. me from its polynomial form: with u = r /
// r^2, sum_lm Qs_lm D_lm(u) = sum_abc P_abc ux^a uy^b uz^c, P_abc = sum_m
// Qs_lm cart[lm][a][b] (l = a + b + c; formed once per pair by
// k_pair_moments, layout mono_k), so v = (1/r) sum P_abc ux^a uy^b uz^c,
// evaluated by nested Horner steps (84 multiply-adds per point).  Double-float
// (mixed form) and FP64 versions.
__device__ __forceinline__ DF me_potential_cart_df(const DF* __restrict__ P, DF x, DF y, DF z) {
  const DF r2 = df_fma(z, z, df_dot2(x, x, y, y));
  const DF ir2 = df_rcp(r2);
  const DF ux = df_mul(x, ir2), uy = df_mul(y, ir2), uz = df_mul(z, ir2);
  DF pa{0.f, 0.f};
#pragma unroll
  for (int a = SEA_LMAX; a >= 0; --a) {
    DF pb{0.f, 0.f};
#pragma unroll
    for (int b = SEA_LMAX - a; b >= 0; --b) {
      DF pc = P[mono_k(a, b, SEA_LMAX - a - b)];
#pragma unroll
      for (int c = SEA_LMAX - a - b - 1; c >= 0; --c) pc = df_fma(pc, uz, P[mono_k(a, b, c)]);
      pb = (b == SEA_LMAX - a) ? pc : df_fma(pb, uy, pc);
    }
    pa = (a == SEA_LMAX) ? pb : df_fma(pa, ux, pb);
  }
  return df_mul(pa, df_sqrt(ir2));
}
__device__ __forceinline__ double me_potential_cart(const double* __restrict__ P, double x,
                                                    double y, double z) {
  const double ir2 = 1.0 / (x * x + y * y + z * z);
  const double ux = x * ir2, uy = y * ir2, uz = z * ir2;
  double pa = 0.0;
#pragma unroll
  for (int a = SEA_LMAX; a >= 0; --a) {
    double pb = 0.0;
#pragma unroll
    for (int b = SEA_LMAX - a; b >= 0; --b) {
      double pc = P[mono_k(a, b, SEA_LMAX - a - b)];
#pragma unroll
      for (int c = SEA_LMAX - a - b - 1; c >= 0; --c) pc = fma(pc, uz, P[mono_k(a, b, c)]);
      pb = (b == SEA_LMAX - a) ? pc : fma(pb, uy, pc);
    }
    pa = (a == SEA_LMAX) ? pb : fma(pa, ux, pb);
  }
  return pa * sqrt(ir2);
}

// harm_accumulate in double-float: acc[q] += w D_q(x, y, z), the same
// recurrences in the same order.
__device__ __forceinline__ void harm_accumulate_df(DF w, DF x, DF y, DF z, DF* acc) {
  const DF r2 = df_fma(z, z, df_dot2(x, x, y, y));
  DF Dm[2 * SEA_LMAX + 1], Dc[2 * SEA_LMAX + 1], Dn[2 * SEA_LMAX + 1];  // l-1, l, l+1
#pragma unroll
  for (int k = 0; k < 2 * SEA_LMAX + 1; ++k) Dm[k] = Dc[k] = Dn[k] = DF{0.f, 0.f};
  Dm[SEA_LMAX] = DF{1.f, 0.f};
  Dc[SEA_LMAX + 1] = x;
  Dc[SEA_LMAX - 1] = y;
  Dc[SEA_LMAX] = z;
  acc[0] = df_add(acc[0], w);
  acc[lmi(1, -1)] = df_fma(w, y, acc[lmi(1, -1)]);
  acc[lmi(1, 0)] = df_fma(w, z, acc[lmi(1, 0)]);
  acc[lmi(1, 1)] = df_fma(w, x, acc[lmi(1, 1)]);
#pragma unroll
  for (int l = 1; l < SEA_LMAX; ++l) {
    Dn[SEA_LMAX + l + 1] = df_dot2(x, Dc[SEA_LMAX + l], df_neg(y), Dc[SEA_LMAX - l]);
    Dn[SEA_LMAX - l - 1] = df_dot2(y, Dc[SEA_LMAX + l], x, Dc[SEA_LMAX - l]);
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      if (m >= -(l - 1) && m <= l - 1) {
        const DF g = df_mul(DF{c_harm.gam_hi[l][m + SEA_LMAX], c_harm.gam_lo[l][m + SEA_LMAX]}, r2);
        Dn[SEA_LMAX + m] = df_dot2(z, Dc[SEA_LMAX + m], df_neg(g), Dm[SEA_LMAX + m]);
      } else {
        Dn[SEA_LMAX + m] = df_mul(z, Dc[SEA_LMAX + m]);
      }
    }
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m)
      acc[lmi(l + 1, m)] = df_fma(w, Dn[SEA_LMAX + m], acc[lmi(l + 1, m)]);
#pragma unroll
    for (int k = 0; k < 2 * SEA_LMAX + 1; ++k) {
      Dm[k] = Dc[k];
      Dc[k] = Dn[k];
    }
  }
}

// Exclusive scan over the CTA of one 64-bit integer per thread (blockDim.x
// a multiple of 32, at most 1024): warp shuffles, then the warp totals by
// the first warp.  Returns this thread's exclusive prefix; *total = the
// CTA's sum in every thread.  `ws` holds 32 values of shared memory.
// Integer sums, so the results equal a serial scan's.
__device__ __forceinline__ long long block_exscan_ll(long long v, long long* ws, long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    long long t = lane < nw ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const long long before = (w ? ws[w - 1] : 0) + x - v;
  *total = ws[nw - 1];
  __syncthreads();  // ws may be reused
  return before;
}
// Maximum over the CTA of one 64-bit integer per thread (same shape rules).
__device__ __forceinline__ long long block_max_ll(long long v, long long* ws) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, v, o);
    v = y > v ? y : v;
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) ws[w] = v;
  __syncthreads();
  long long m = ws[0];
  for (int k = 1; k < nw; ++k) m = ws[k] > m ? ws[k] : m;
  __syncthreads();
  return m;
}

// Sum over the block of one double; every thread gets the same total, added
// in a fixed order (lane tree, then warps in index order).  `slots` holds
// 32 doubles of shared memory, reused only after the next __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* slots) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) slots[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; ++k) s += slots[k];
  return s;
}

}  // namespace sea

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

struct SeaBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

namespace sea {

// Grid tiles of the ACE contractions: 8 x 4 x 4 points, point r of a tile
// at x = r % 8, y = (r / 8) % 4, z = r / 32 inside it.
#define TX 8
#define TY 4
#define TZ 4
#define TP (TX * TY * TZ)

struct TileGeom {
  int nx, ny, nz, ntx, nty, ntz;
};

// Flat grid index of point r of tile T (-1 outside the grid).
__device__ __forceinline__ long long tile_point(const TileGeom& G, int T, int r) {
  const int txi = T % G.ntx, tyi = (T / G.ntx) % G.nty, tzi = T / (G.ntx * G.nty);
  const int x = txi * TX + (r % TX), y = tyi * TY + (r / TX) % TY, z = tzi * TZ + r / (TX * TY);
  if (x >= G.nx || y >= G.ny || z >= G.nz) return -1;
  return ((long long)z * G.ny + y) * G.nx + x;
}

inline TileGeom make_tile_geom(const int N[3]) {
  TileGeom G;
  G.nx = N[0];
  G.ny = N[1];
  G.nz = N[2];
  G.ntx = (G.nx + TX - 1) / TX;
  G.nty = (G.ny + TY - 1) / TY;
  G.ntz = (G.nz + TZ - 1) / TZ;
  return G;
}

}  // namespace sea

// A launch sequence recorded into a CUDA graph: the executable graph, the
// signature (sizes, parameters, buffer addresses) it was recorded with, and
// the number of kernels in it.
struct LaunchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> sig;
  long long launches = 0;
};

struct sea_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  double cell[3] = {0, 0, 0};
  int N[3] = {0, 0, 0};
  double h[3] = {0, 0, 0};
  double dV = 0;
  size_t ng = 0;
  sea_params prm{};
  double w_ax[3][SEA_FDP + 1];  // -c_k / h_a^2 (negated second-difference weights)
  double w_center = 0;          // -sum_a c_0 / h_a^2

  bool poisoned = false;
  char err[256] = {0};

  int n_orb = 0;
  bool have_phi = false, have_vxx = false, have_ace = false, apply_timed = false;
  bool ace_eigen = false, w_dense = false;
  void* batch_cache = nullptr;  // CUDA graph of sea_apply_vxx_batch (batch.cu)
  SeaBuf bdesc, bitems;

  // plan sizes (host copies)
  int P = 0, Pproto = 0, E = 0;
  long long U = 0, WC = 0, max_window = 0;
  int cg_pad_max = 0;  // largest zero-padded pair box (floats), for the mixed CG

  sea_stats stats{};

  // device buffers
  SeaBuf phi, vxx_dev, psi_dev, out_dev;
  SeaBuf rowsum, colsum, marg, box;
  SeaBuf cand_flag, cand_geom, list_a, list_b, cand_S, counts;
  SeaBuf pinfo, pS, psize, voff, order, Q, epair, iters;
  SeaBuf vbuf, bbuf, rbuf, pbuf, qbuf;
  SeaBuf eptr, eent, ewin, coff, cbuf;
  SeaBuf status, exx_dev, queue;
  SeaBuf onorm;  // per-orbital partial sums of phi^2 (input check of sea_set_orbitals)
  // ACE
  SeaBuf wdig;  // the mixed form's W digits (tensor-core contraction)
  SeaBuf wx;    // the mixed form's per-tile W digit images (tensor-core expansion)
  SeaBuf xevb;  // the expansion's H exponents per (tile, vector)
  SeaBuf gbuf;  // ghost (boundary) values of the pair boxes, 36 voff per pair
  SeaBuf flowbuf;  // the mixed form's one-launch Cholesky chain: DF blocks and task flags
  SeaBuf scdm_u, scdm_c;  // SCDM rotation and pivots
  SeaBuf tmask, tptr_o, tlist_o, tslot_o, tptr_t, tlist_t, partial, Mbuf, Abuf, Lbuf, Linv,
      Gbuf, Hbuf, Hbuf2;
  int n_tiles = 0, tile_inc = 0, max_tile_list = 0;
  long long list_cap = 1;    // entries per list array (the second array's offset)
  bool lists_ready = false;  // the tile lists of the last plan's W support are formed
                             // and their counts on the host

  long long launches = 0;
  cudaEvent_t ev[16] = {};
  // host-buffer transfers: copy streams (host to device, device to host) and
  // per-chunk events, created with the context
  cudaStream_t xfer[2] = {};
  std::vector<int> h_eptr;  // entry offsets per orbital, host copy (last plan)
  struct sea_unet* unet = nullptr;  // learned warm start (attached model, not owned)
  bool cg_warm = false;             // the next CG starts from the guess in vbuf
  LaunchGraph g_chol;  // the Cholesky / L^-1 / E_xx^ACE chain
  LaunchGraph g_plan;  // the plan (boxes, pairs, accumulation entries)
  bool far_side = false;            // the contributions outside the pair boxes were
                                    // launched on xfer[0] (done at xev[1])
  cudaEvent_t xev[2 * SEA_XCHUNKS_MAX + 2] = {};
};
// enqueue() issues a fixed launch sequence on c->stream.  On a stream that
// can be captured it is recorded once into gc (again whenever sig changes)
// and the graph is replayed, which removes most of the gaps between short
// dependent launches; on the legacy stream it runs directly.  enqueue()
// must not allocate or synchronise.
template <class F>
inline cudaError_t run_graph(sea_ctx* c, LaunchGraph& gc, const std::vector<uintptr_t>& sig,
                             F enqueue) {
  if (!c->stream) return enqueue();
  if (!gc.exec || gc.sig != sig) {
    if (gc.exec) {
      cudaGraphExecDestroy(gc.exec);
      gc.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long long l0 = c->launches;
    e = enqueue();
    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    gc.launches = c->launches - l0;
    c->launches = l0;
    gc.sig = sig;
  }
  c->launches += gc.launches;
  return cudaGraphLaunch(gc.exec, c->stream);
}


// Host-side helpers implemented in api.cu.
sea_status sea_fail(sea_ctx* c, sea_status s, const char* msg);
void sea_batch_cache_free(sea_ctx* c);
bool sea_ensure(sea_ctx* c, SeaBuf& b, size_t bytes);

// Pair record (device), one per selected pair, in (i, j) order.
struct PairInfo {
  int i, j;
  int lo[3], ext[3], k[3];
  int n;  // ext[0]*ext[1]*ext[2]
};

// Accumulation entry (Eq. tDxx): orbital o receives v_pair * phi_partner on
// the window [ws, ws + wl) (unwrapped grid coordinates, pair frame).
struct Entry {
  int pair, o, partner;
  int ws[3], wl[3];
};

namespace sea {
// Window points per unit of the far-field work (k_contrib's CTAs and the
// mixed CG's far-field items).
#define SEA_CHUNK 1024

// q = floor(a / d) and *r = a - q d for 0 <= a < 2^24, 1 <= d < 2^24: the
// FP32 product a (1/d) is within (a/d) 2^-23 < 1 of a/d, so its truncation
// is q or q +- 1, corrected once by the sign and size of the remainder.
__host__ __device__ __forceinline__ int divmod_small(int a, int d, int* r) {
  int q = (int)((float)a * (1.0f / (float)d));
  int rr = a - q * d;
  if (rr < 0) {
    --q;
    rr += d;
  } else if (rr >= d) {
    ++q;
    rr -= d;
  }
  *r = rr;
  return q;
}

// The pair box in the coordinates of an entry's window, clipped to it:
// [b0[a], b1[a]) per axis, n_in points inside and n_out outside.  An empty
// intersection is kept as the empty box [0, 0)^3, so that every window point
// falls in the "z above" part of window_outside_point.
struct WinSplit {
  int b0[3], b1[3];
  int n_in, n_out;
};
__host__ __device__ __forceinline__ WinSplit window_split(const Entry& e, const PairInfo& P) {
  WinSplit s;
  bool empty = false;
  for (int a = 0; a < 3; ++a) {
    const int lo = P.lo[a] - e.ws[a], hi = lo + P.ext[a];
    s.b0[a] = lo < 0 ? 0 : (lo > e.wl[a] ? e.wl[a] : lo);
    s.b1[a] = hi < 0 ? 0 : (hi > e.wl[a] ? e.wl[a] : hi);
    empty = empty || s.b0[a] >= s.b1[a];
  }
  if (empty)
    for (int a = 0; a < 3; ++a) s.b0[a] = s.b1[a] = 0;
  s.n_in = (s.b1[0] - s.b0[0]) * (s.b1[1] - s.b0[1]) * (s.b1[2] - s.b0[2]);
  s.n_out = e.wl[0] * e.wl[1] * e.wl[2] - s.n_in;
  return s;
}

// Window coordinates of point u (0 <= u < n_out, n_out < 2^24) of the window
// points outside the pair box, numbered through six disjoint boxes: the
// planes below and above the box's z range, then within that z range the
// rows below and above its y range, then within that y range the runs left
// and right of its x range; x fastest inside each.
__host__ __device__ __forceinline__ void window_outside_point(const WinSplit& s, const int wl[3],
                                                              int u, int* tx, int* ty, int* tz) {
  const int wx = wl[0], wy = wl[1], wz = wl[2];
  const int zb = s.b1[2] - s.b0[2], yb = s.b1[1] - s.b0[1];
  const int n1 = s.b0[2] * wx * wy, n2 = (wz - s.b1[2]) * wx * wy;
  const int n3 = zb * s.b0[1] * wx, n4 = zb * (wy - s.b1[1]) * wx, n5 = zb * yb * s.b0[0];
  int ox = 0, oy = 0, oz = 0, bx = wx, by = wy;
  if (u < n1) {
  } else if ((u -= n1) < n2) {
    oz = s.b1[2];
  } else if ((u -= n2) < n3) {
    oz = s.b0[2];
    by = s.b0[1];
  } else if ((u -= n3) < n4) {
    oz = s.b0[2];
    oy = s.b1[1];
    by = wy - s.b1[1];
  } else if ((u -= n4) < n5) {
    oz = s.b0[2];
    oy = s.b0[1];
    by = yb;
    bx = s.b0[0];
  } else {
    u -= n5;
    oz = s.b0[2];
    oy = s.b0[1];
    by = yb;
    ox = s.b1[0];
    bx = wx - s.b1[0];
  }
  int rx, ry;
  const int q = divmod_small(u, bx, &rx);
  const int qz = divmod_small(q, by, &ry);
  *tx = ox + rx;
  *ty = oy + ry;
  *tz = oz + qz;
}

// Window contributions c = v phi_partner (Eq. tDxx) of entry e (window-
// compact output out[t], t = (tz wy + ty) wx + tx): v is the pair's CG
// solution (v, box layout) inside the pair box and the multipole potential
// (coefficients Pd, double-float, or Ps, FP64) outside.  part 0: every
// window point, t = t0 + threadIdx.x, + blockDim.x, ... < t1; 1: only the
// points outside the box (they need the moments alone), 2: only those
// inside (they need the solution); for parts 1 and 2 with compact set, t0
// and t1 number the points of that part alone (window_outside_point; the
// box's points in x-fastest order), so that no lane idles on a point of the
// other part, else they are window points and the other part's are skipped.
// DFM: double-float products (mixed form), else FP64.
template <bool DFM>
__device__ __forceinline__ void contrib_range(int part, bool compact, const WinSplit& sp,
                                              const Entry& e, const PairInfo& P,
                                              const double* __restrict__ phi, int nx, int ny,
                                              int nz, const double* __restrict__ v, const DF* Pd,
                                              const double* Ps, double hx, double hy, double hz,
                                              double* __restrict__ out, int t0, int t1) {
  const DF Hx = df_from_double(hx), Hy = df_from_double(hy), Hz = df_from_double(hz);
  const size_t ng = (size_t)nx * ny * nz;
  const double* fp = phi + (size_t)e.partner * ng;
  const double cx = 0.5 * (P.ext[0] - 1), cy = 0.5 * (P.ext[1] - 1), cz = 0.5 * (P.ext[2] - 1);
  const float cxf = 0.5f * i2f_exact(P.ext[0] - 1), cyf = 0.5f * i2f_exact(P.ext[1] - 1),
              czf = 0.5f * i2f_exact(P.ext[2] - 1);
  const int wx = e.wl[0], wy = e.wl[1];
  const int gx0 = wrapi(e.ws[0], nx), gy0 = wrapi(e.ws[1], ny), gz0 = wrapi(e.ws[2], nz);
  const int S = blockDim.x;
  // one window point (tx, ty, tz): its value into out[(tz wy + ty) wx + tx]
  auto point = [&](int tx, int ty, int tz, bool inside) {
    const int lx = e.ws[0] + tx - P.lo[0], ly = e.ws[1] + ty - P.lo[1], lz = e.ws[2] + tz - P.lo[2];
    int gx = gx0 + tx, gy = gy0 + ty, gz = gz0 + tz;  // window lengths are at most n
    gx -= gx >= nx ? nx : 0;
    gy -= gy >= ny ? ny : 0;
    gz -= gz >= nz ? nz : 0;
    const size_t g = ((size_t)gz * ny + gy) * nx + gx;
    const int t = (tz * wy + ty) * wx + tx;
    if (DFM) {  // c = v phi in double-float, no FP64 instruction
      DF val;
      if (inside) {
        const float2 s = split64(v[(lz * P.ext[1] + ly) * P.ext[0] + lx]);
        val = DF{s.x, s.y};
      } else {  // lx - cx etc. are half-integers, exact in FP32
        val = me_potential_cart_df(Pd, df_mul_f(i2f_exact(lx) - cxf, Hx),
                                   df_mul_f(i2f_exact(ly) - cyf, Hy), df_mul_f(i2f_exact(lz) - czf, Hz));
      }
      const float2 f = split64(fp[g]);
      out[t] = df_to_double(df_mul(val, DF{f.x, f.y}));
    } else {
      const double val = inside ? v[(lz * P.ext[1] + ly) * P.ext[0] + lx]
                                : me_potential_cart(Ps, (lx - cx) * hx, (ly - cy) * hy, (lz - cz) * hz);
      out[t] = __dmul_rn(val, fp[g]);
    }
  };
  // parts 0 and 2, and part 1 without compact: a box [ox, ox + bx) x
  // [oy, oy + by) x ... (the window, or with compact part 2 the pair box
  // within it) walked with (kx, ky, kz) advanced by the CTA stride without
  // divisions; compact part 1: window_outside_point
  const bool outer = compact && part == 1, box = compact && part == 2;
  const int ox = box ? sp.b0[0] : 0, oy = box ? sp.b0[1] : 0, oz = box ? sp.b0[2] : 0;
  const int bx = box ? sp.b1[0] - sp.b0[0] : wx, by = box ? sp.b1[1] - sp.b0[1] : wy;
  const int bxy = bx * by;
  const int dz = S / bxy, dy = (S - dz * bxy) / bx, dx = S - dz * bxy - dy * bx;
  int kz = (t0 + (int)threadIdx.x) / bxy;
  int ky = (t0 + (int)threadIdx.x - kz * bxy) / bx;
  int kx = t0 + (int)threadIdx.x - kz * bxy - ky * bx;
  if (box) {
    // in-box points: the loop is bound by the latency of its two loads per
    // point, so each thread takes CU points (t, t + S, ...) with all their
    // loads issued before the first product; the products are those of
    // `point`, so the results are the same bits
    constexpr int CU = 4;
    const int l0 = e.ws[0] - P.lo[0], l1 = e.ws[1] - P.lo[1], l2 = e.ws[2] - P.lo[2];
    for (int t = t0 + threadIdx.x; t < t1; t += CU * S) {
      int lq[CU], tq[CU];
      size_t gq[CU];
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int tx = ox + kx, ty = oy + ky, tz = oz + kz;
        kx += dx;
        ky += dy;
        kz += dz;
        if (kx >= bx) {
          kx -= bx;
          ++ky;
        }
        if (ky >= by) {
          ky -= by;
          ++kz;
        }
        int gx = gx0 + tx, gy = gy0 + ty, gz = gz0 + tz;
        gx -= gx >= nx ? nx : 0;
        gy -= gy >= ny ? ny : 0;
        gz -= gz >= nz ? nz : 0;
        gq[u] = ((size_t)gz * ny + gy) * nx + gx;
        tq[u] = (tz * wy + ty) * wx + tx;
        lq[u] = ((l2 + tz) * P.ext[1] + (l1 + ty)) * P.ext[0] + (l0 + tx);
      }
      double vq[CU], fq[CU];
#pragma unroll
      for (int u = 0; u < CU; ++u)
        if (t + u * S < t1) {
          vq[u] = v[lq[u]];
          fq[u] = fp[gq[u]];
        }
#pragma unroll
      for (int u = 0; u < CU; ++u)
        if (t + u * S < t1) {
          if (DFM) {
            const float2 s = split64(vq[u]), f = split64(fq[u]);
            out[tq[u]] = df_to_double(df_mul(DF{s.x, s.y}, DF{f.x, f.y}));
          } else {
            out[tq[u]] = __dmul_rn(vq[u], fq[u]);
          }
        }
    }
    return;
  }
  for (int t = t0 + threadIdx.x; t < t1; t += S) {
    int tx, ty, tz;
    bool inside = box;
    if (outer) {
      window_outside_point(sp, e.wl, t, &tx, &ty, &tz);
    } else {
      tx = ox + kx;
      ty = oy + ky;
      tz = oz + kz;
      kx += dx;
      ky += dy;
      kz += dz;
      if (kx >= bx) {
        kx -= bx;
        ++ky;
      }
      if (ky >= by) {
        ky -= by;
        ++kz;
      }
      if (!box) {
        const int lx = e.ws[0] + tx - P.lo[0], ly = e.ws[1] + ty - P.lo[1],
                  lz = e.ws[2] + tz - P.lo[2];
        inside = lx >= 0 && lx < P.ext[0] && ly >= 0 && ly < P.ext[1] && lz >= 0 && lz < P.ext[2];
        if ((part == 1 && inside) || (part == 2 && !inside)) continue;
      }
    }
    point(tx, ty, tz, inside);
  }
}


// Launch wrappers (each file implements its own).
cudaError_t launch_plan_boxes(sea_ctx* c);
cudaError_t launch_plan_pairs(sea_ctx* c);
cudaError_t launch_pair_setup(sea_ctx* c);
cudaError_t launch_cg(sea_ctx* c);
cudaError_t launch_contrib_far(sea_ctx* c, cudaEvent_t setup_done);
// chol_flow.cu: the mixed form's Cholesky of -Mbar, L^-1 and E_xx^ACE in one
// cooperative launch (scratch of chol_flow_bytes(n) bytes).
size_t chol_flow_bytes(int n);
cudaError_t launch_chol_flow(cudaStream_t st, int device, const double* M, int n, double* L,
                             double* Linv, void* scratch, unsigned* status, double* exx);
void make_batch_desc(sea_ctx* c, void* out);
size_t batch_desc_bytes();
// The persistent batched CG: ctas_per_sm CTAs per SM (0 or above the
// occupancy limit: the limit).
cudaError_t launch_cg_batch(cudaStream_t st, int device, const void* descs, const int2* items,
                            int total, int* queue, int pad_cap, bool mixed, int ctas_per_sm);
int cg_batch_max_ctas_per_sm(int device, int pad_cap, bool mixed);
int cg_pad_cap(const sea_ctx* c);
cudaError_t launch_entries(sea_ctx* c);
// V_xx phi into out (the context's W) and, when out2 is not null, also into
// out2 (the caller's device buffer), both written by the same stores.
cudaError_t launch_accumulate(sea_ctx* c, double* out, double* out2 = nullptr,
                              bool with_exx = true);
cudaError_t launch_accumulate_range(sea_ctx* c, double* out, int o_begin, int o_end, int e_begin,
                                    int e_end, double* out2 = nullptr);
cudaError_t launch_exx(sea_ctx* c, cudaStream_t st);
// Learned warm start (unet.cu): x0 of every pair's CG from the attached model.
cudaError_t launch_warm_start(sea_ctx* c);
// SCDM localization of the orbitals in the context (scdm.cu): U and the
// pivots on the device; the localized orbitals replace c->phi.
cudaError_t launch_scdm(sea_ctx* c, double* U_dev, long long* C_dev);
// Damped Jacobi sweeps on every pair's starting vector (pair.cu).
cudaError_t launch_smooth(sea_ctx* c, int sweeps, double omega);
// Mixed form's contraction with W on the tensor cores.  launch_w_digits
// splits W's rows on every tile of every list once into wbuf
// (w_digits_bytes(slots), slots = total list length); launch_gram_tc then
// forms partial[slot m + a] for A's m rows.  *queue is reset on the stream.
size_t w_digits_bytes(long long slots);
cudaError_t launch_w_digits(cudaStream_t st, const double* W, const TileGeom& G, size_t ng,
                            int n_tiles, int max_list, const int* tptr, const int* tlist,
                            long long slots, void* wbuf);
size_t wx_digits_bytes(int n_tiles, long long slots);
cudaError_t launch_wx_digits(cudaStream_t st, const double* W, const TileGeom& G, size_t ng,
                             int n_tiles, const int* tptr, const int* tlist, const int* tsub,
                             void* wxbuf);
cudaError_t launch_expand_tc(cudaStream_t st, int device, const void* wxbuf, const TileGeom& G,
                             size_t ng, int n_tiles, const int* tptr, const int* tlist,
                             const double* H, long long hj, long long hv, int m, bool negate,
                             double* out, int* evbuf, int* queue, unsigned* status);
int expand_tc_max_list();
cudaError_t launch_gram_tc(cudaStream_t st, int device, const double* A, int m, const TileGeom& G,
                           size_t ng, int n_tiles, const int* tptr, long long slots,
                           const void* wbuf, double* partial, int* queue, unsigned* status);
cudaError_t launch_ace_lists(sea_ctx* c, cudaStream_t st);
cudaError_t launch_ace_build(sea_ctx* c);
cudaError_t launch_ace_eigen(sea_ctx* c);
cudaError_t launch_ace_apply(sea_ctx* c, const double* psi, int n_vec, double* out);
cudaError_t launch_ace_vectors(sea_ctx* c, double* xi);
cudaError_t upload_harmonics_pair();
void fornberg_weights(double* w);
cudaError_t launch_cg_boxes(cudaStream_t stream, int device, const double h[3], int nbox,
                            const PairInfo* boxes, const long long* voff, const int* order,
                            const double* rhs, double* x, double* r, double* p, double* q,
                            int* iters, unsigned* status, int* queue, double tol, int tol_mode,
                            int max_iter);
cudaError_t upload_harmonics_accum();
}  // namespace sea
