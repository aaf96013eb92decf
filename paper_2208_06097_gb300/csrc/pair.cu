// pair.cu -- per-pair Poisson problems (Sec. II B: Eqs. pe, me, mepole).
//
// k_pair_moments (one CTA per pair): rho_ij = phi_i phi_j on Omega_ij and
//   its multipole moments about the box centre; b = 4 pi rho.
// k_ghost_eval (one CTA per pair and axis), k_boundary_apply (one CTA per
//   pair): the multipole potential at every point outside the box that the
//   37-point stencil reaches (one coordinate outside, by 1..6), added to b
//   with the stencil weights.
// k_cg (persistent, longest pairs first): conjugate gradients for
//   -Lap_h v = b on the box with zero values outside, FP64, two block
//   reductions per iteration (warp shuffles, then warps in fixed order),
//   the 37-point O(h^12) operator written as 37 fused multiply-adds (on this
//   part the FP64 FMA pipe issues faster than FP64 add); then the pair
//   integral sum rho v dV of Eq. exxGen_mlwf.
#include <cstring>

#include "sea_internal.cuh"

namespace sea {

struct StencilW {
  double ax[3][SEA_FDP + 1];  // -c_k / h_a^2
  double center;              // -sum_a c_0 / h_a^2
  double rhs[3][SEA_FDP + 1]; // +c_k / h_a^2 (boundary values moved to b)
};

// Pair density and moments, one CTA per pair: b = 4 pi rho on the box,
// Qs = rescaled multipole moments of rho about the box centre (Eq. mepole),
//   Qs_lm = kappa_lm^2 dV sum_r rho(r) D_lm(r).
// D_lm is a homogeneous polynomial of degree l (the coefficients cart[lm]
// expanded from the harmonic recurrence), so the sum is a fixed combination
// of the Cartesian moments M_abc = sum_r rho x^a y^b z^c, a + b + c <= 6,
// which on the box grid separate.  With the point's offsets from the box
// centre in half grid steps, u = 2 x - (ex - 1) (v, w likewise; x = u hx / 2),
//   S_a(y, z) = sum_x rho u^a                (one thread per row),
//   T_ab(z)   = sum_y v^b S_a(y, z)          (a + b <= 6, per slab of planes),
//   M_abc     = (hx/2)^a (hy/2)^b (hz/2)^c sum_z w^c T_ab(z),
// all sums in a fixed order.  Per point this is 7 products and sums instead
// of the 49-term harmonic recurrence.  DFM: rho and S, T, M in double-float
// arithmetic (mixed form), else FP64; the last combination in FP64.
namespace {
template <bool DFM>
struct MomR;  // the accumulation type and its operations
template <>
struct MomR<true> {
  typedef DF T;
  static __device__ __forceinline__ T zero() { return DF{0.f, 0.f}; }
  static __device__ __forceinline__ T mul_i(T a, int k) { return df_mul_f(i2f_exact(k), a); }
  static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T prod(double a, double c) {
    const float2 as = split64(a), cs = split64(c);
    return df_mul(DF{as.x, as.y}, DF{cs.x, cs.y});
  }
  static __device__ __forceinline__ T one() { return DF{1.f, 0.f}; }
  static __device__ __forceinline__ double to_double(T a) { return df_to_double(a); }
};
template <>
struct MomR<false> {
  typedef double T;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T mul_i(T a, int k) { return a * (double)k; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T prod(double a, double c) { return a * c; }
  static __device__ __forceinline__ T one() { return 1.0; }
  static __device__ __forceinline__ double to_double(T a) { return a; }
};
constexpr int MOM_E = SEA_LMAX + 1;                       // powers 0..6
constexpr int MOM_NAB = MOM_E * (MOM_E + 1) / 2;           // 28 pairs a + b <= 6
constexpr int MOM_NABC = MOM_E * (MOM_E + 1) * (MOM_E + 2) / 6;  // 84 monomials
constexpr int MOM_ZSLAB = 16;                             // planes per slab at most
// (a, b) of pair index k (a + b <= 6, a-major)
__device__ __forceinline__ void mom_ab(int k, int* a, int* b) {
  int aa = 0;
  while (k >= MOM_E - aa) {
    k -= MOM_E - aa;
    ++aa;
  }
  *a = aa;
  *b = k;
}
__device__ __forceinline__ int mom_abi(int a, int b) { return a * MOM_E - a * (a - 1) / 2 + b; }
}  // namespace

// Dynamic shared memory of k_pair_moments for a grid with ny, nz points on
// the y and z axes (box extents are at most those).
size_t pair_moments_smem(int ny, int nz) {
  const size_t rows = (size_t)std::max(256, ny);
  return (rows * MOM_E + (size_t)MOM_ZSLAB * MOM_NAB + (size_t)(ny + nz) * MOM_E) * 8 +
         (size_t)MOM_NABC * 8;
}

template <bool DFM>
__global__ void __launch_bounds__(256)
    k_pair_moments(const double* __restrict__ phi, int nx, int ny, int nz,
                   const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff,
                   double hx, double hy, double hz, double dV, int lmax,
                   double* __restrict__ bbuf, double* __restrict__ Qout,
                   const int* __restrict__ order) {
  typedef MomR<DFM> R;
  typedef typename R::T T;
  extern __shared__ double mom_sm[];
  const int p = order[blockIdx.x];  // the largest pairs first: the small ones fill the tail
  const PairInfo P = pinfo[p];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2];
  const int Z = min(MOM_ZSLAB, max(1, 256 / ey));  // planes per slab
  T* S = reinterpret_cast<T*>(mom_sm);             // [rows of the slab][7]
  T* Tz = S + (size_t)max(256, ey) * MOM_E;        // [Z][28]
  T* vp = Tz + MOM_ZSLAB * MOM_NAB;                // [ey][7]: v^b
  T* wp = vp + (size_t)ey * MOM_E;                 // [ez][7]: w^c
  double* Mf = reinterpret_cast<double*>(wp + (size_t)ez * MOM_E);  // [84]
  const size_t ng = (size_t)nx * ny * nz;
  const double* fi = phi + (size_t)P.i * ng;
  const double* fj = phi + (size_t)P.j * ng;
  double* b = bbuf + voff[p];
  const double fourpi = 4.0 * 3.14159265358979323846;
  // powers of the half-step offsets along y and z
  for (int k = threadIdx.x; k < ey + ez; k += blockDim.x) {
    const bool isy = k < ey;
    const int i = isy ? k : k - ey, e = isy ? ey : ez;
    const int o = 2 * i - (e - 1);
    T* dst = (isy ? vp : wp) + (size_t)i * MOM_E;
    T pw = R::one();
    for (int c = 0; c < MOM_E; ++c) {
      dst[c] = pw;
      pw = R::mul_i(pw, o);
    }
  }
  // this thread's monomial of M (threads 0..83)
  int ma = 0, mb = 0, mc = 0;
  if (threadIdx.x < MOM_NABC) {
    int k = threadIdx.x, l = 0;
    while (k >= (l + 1) * (l + 2) / 2) {
      k -= (l + 1) * (l + 2) / 2;
      ++l;
    }
    ma = 0;  // degree l: (a, b) with a + b <= l in a-major order, c = l - a - b
    while (k >= l - ma + 1) {
      k -= l - ma + 1;
      ++ma;
    }
    mb = k;
    mc = l - ma - mb;
  }
  T macc = R::zero();
  const int gx0 = wrapi(P.lo[0], nx);
  for (int z0 = 0; z0 < ez; z0 += Z) {
    const int zn = min(Z, ez - z0), rows = zn * ey;
    __syncthreads();  // S, Tz of the previous slab are consumed; the powers are in place
    // S_a(y, z): one thread per row; b = 4 pi rho on the way
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const int y = r % ey, z = z0 + r / ey;
      const size_t rowg =
          ((size_t)wrapi(P.lo[2] + z, nz) * ny + wrapi(P.lo[1] + y, ny)) * nx;
      double* brow = b + ((size_t)z * ey + y) * ex;
      T s[MOM_E];
#pragma unroll
      for (int a = 0; a < MOM_E; ++a) s[a] = R::zero();
      int gx = gx0;
      for (int x = 0; x < ex; ++x) {
        const double av = fi[rowg + gx], cv = fj[rowg + gx];
        brow[x] = fourpi * (av * cv);
        T pk = R::prod(av, cv);
        const int u = 2 * x - (ex - 1);
        s[0] = R::add(s[0], pk);
#pragma unroll
        for (int a = 1; a < MOM_E; ++a) {
          pk = R::mul_i(pk, u);
          s[a] = R::add(s[a], pk);
        }
        if (++gx == nx) gx = 0;
      }
#pragma unroll
      for (int a = 0; a < MOM_E; ++a) S[(size_t)r * MOM_E + a] = s[a];
    }
    __syncthreads();
    // T_ab(z) for the slab's planes
    for (int it = threadIdx.x; it < zn * MOM_NAB; it += blockDim.x) {
      const int zl = it / MOM_NAB;
      int a, bb;
      mom_ab(it - zl * MOM_NAB, &a, &bb);
      T t = R::zero();
      for (int y = 0; y < ey; ++y)
        t = R::add(t, R::mul(vp[(size_t)y * MOM_E + bb], S[((size_t)zl * ey + y) * MOM_E + a]));
      Tz[zl * MOM_NAB + mom_abi(a, bb)] = t;
    }
    __syncthreads();
    // M_abc += sum over the slab's planes of w^c T_ab(z)
    if (threadIdx.x < MOM_NABC)
      for (int zl = 0; zl < zn; ++zl)
        macc = R::add(macc, R::mul(wp[(size_t)(z0 + zl) * MOM_E + mc], Tz[zl * MOM_NAB + mom_abi(ma, mb)]));
  }
  if (threadIdx.x < MOM_NABC) {
    double sc = R::to_double(macc);
    for (int k = 0; k < ma; ++k) sc *= 0.5 * hx;
    for (int k = 0; k < mb; ++k) sc *= 0.5 * hy;
    for (int k = 0; k < mc; ++k) sc *= 0.5 * hz;
    Mf[threadIdx.x] = sc;
  }
  __syncthreads();
  __shared__ double Qsm[SEA_NQ];
  double* Qp = Qout + (size_t)p * SEA_QSTRIDE;
  if (threadIdx.x < SEA_NQ) {
    const int q = threadIdx.x;
    int l = 0;
    while ((l + 1) * (l + 1) <= q) ++l;
    double s = 0.0;
    const int base = l * (l + 1) * (l + 2) / 6;  // monomials of lower degree
    int k = 0;
    for (int a = 0; a <= l; ++a)
      for (int bb = 0; a + bb <= l; ++bb, ++k) s = fma(c_harm.cart[q][a][bb], Mf[base + k], s);
    const double Q = (l <= lmax) ? c_harm.kap2[q] * s * dV : 0.0;
    Qsm[q] = Q;
    Qp[q] = Q;
  }
  __syncthreads();
  // the potential's coefficients P_abc = sum_m Qs_lm cart[lm][a][b], l = a + b + c
  if (threadIdx.x < MOM_NABC) {
    const int l = ma + mb + mc;
    double s = 0.0;
    for (int m = -l; m <= l; ++m) s = fma(Qsm[lmi(l, m)], c_harm.cart[lmi(l, m)][ma][mb], s);
    Qp[SEA_NQ + mono_k(ma, mb, mc)] = s;
  }
}

// Boundary values (Eq. me) at every point outside the box that the
// 37-point stencil reaches, moved into b with the stencil weights, in two
// kernels.  k_ghost_eval (a CTA per pair and axis, the largest pairs first):
// the ghost values of every line across the axis (one evaluation per
// thread) into a global buffer, per pair at 36 voff (12 values per line;
// the three faces, each at most the box's volume, fit in 36 times it).
// k_boundary_apply (a CTA per pair): one thread per (line, boundary point)
// adds the weighted ghost values into b, the axes one after the other, so
// every b entry is updated in a fixed order.
// The stencil's right-hand-side weights as double-float pairs (mixed form).
struct StencilWd {
  float hi[3][SEA_FDP + 1], lo[3][SEA_FDP + 1];
};

// Line (u1, u2) across axis a: its coordinates on the other two axes, the
// face extents and the ghost buffer offset of axis a within the pair.
__device__ __forceinline__ void ghost_face(int a, int ex, int ey, int ez, int* e1, int* e2,
                                           int* ea, int* sa, int* goff) {
  *e1 = a == 0 ? ey : ex;
  *e2 = a == 2 ? ey : ez;
  *ea = a == 0 ? ex : (a == 1 ? ey : ez);
  *sa = a == 0 ? 1 : (a == 1 ? ex : ex * ey);
  *goff = 2 * SEA_FDP * (a == 0 ? 0 : (a == 1 ? ey * ez : ey * ez + ex * ez));
}

// DFM: the potentials in double-float arithmetic (mixed form; four CTAs per
// SM, the nested Horner steps being one dependent chain per point).
template <bool DFM>
__global__ void __launch_bounds__(256, DFM ? 4 : 1)
    k_ghost_eval(const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff,
                 double hx, double hy, double hz, const double* __restrict__ Qg,
                 double* __restrict__ gbuf, const int* __restrict__ order) {
  const int a = blockIdx.x;
  const int p = order[blockIdx.y];  // the largest pairs first: the small ones fill the tail
  const PairInfo P = pinfo[p];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2];
  __shared__ double Ps[SEA_NMONO];
  __shared__ DF Pd[SEA_NMONO];
  if (threadIdx.x < SEA_NMONO) {
    const double q = Qg[(size_t)p * SEA_QSTRIDE + SEA_NQ + threadIdx.x];
    if (DFM)
      Pd[threadIdx.x] = df_from_double(q);
    else
      Ps[threadIdx.x] = q;
  }
  __syncthreads();
  // the potential at grid offsets (ox, oy, oz) from the box centre, in
  // units of h (half-integers, exact in FP32)
  const DF Hx = df_from_double(hx), Hy = df_from_double(hy), Hz = df_from_double(hz);
  const float cx = 0.5f * i2f_exact(ex - 1), cy = 0.5f * i2f_exact(ey - 1),
              cz = 0.5f * i2f_exact(ez - 1);
  constexpr int NG = 2 * SEA_FDP;  // ghost values per line: d = 1..FDP below, then above
  int e1, e2, ea, sa, goff;
  ghost_face(a, ex, ey, ez, &e1, &e2, &ea, &sa, &goff);
  const float ca = a == 0 ? cx : (a == 1 ? cy : cz);
  double* G = gbuf + 36 * voff[p] + goff;
  const int nl = e1 * e2;
  for (int e = threadIdx.x; e < nl * NG; e += blockDim.x) {
    const int line = e / NG, k = e % NG;
    const int u1 = line % e1, u2 = line / e1;
    const float o1 = i2f_exact(u1) - (a == 0 ? cy : cx), o2 = i2f_exact(u2) - (a == 2 ? cy : cz);
    const int d = k % SEA_FDP + 1;
    const float t = i2f_exact(k < SEA_FDP ? -d : ea - 1 + d) - ca;
    const float ox = a == 0 ? t : o1, oy = a == 0 ? o1 : (a == 1 ? t : o2);
    const float oz = a == 2 ? t : o2;
    if (DFM) {
      const DF g = me_potential_cart_df(Pd, df_mul_f(ox, Hx), df_mul_f(oy, Hy), df_mul_f(oz, Hz));
      reinterpret_cast<DF*>(G)[e] = g;
    } else {
      G[e] = me_potential_cart(Ps, (double)ox * hx, (double)oy * hy, (double)oz * hz);
    }
  }
}

template <bool DFM>
__global__ void __launch_bounds__(256)
    k_boundary_apply(const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff,
                     StencilW W, StencilWd Wd, const double* __restrict__ gbuf,
                     double* __restrict__ bbuf, const int* __restrict__ order) {
  const int p = order[blockIdx.x];
  const PairInfo P = pinfo[p];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2];
  double* b = bbuf + voff[p];
  constexpr int NG = 2 * SEA_FDP;
  for (int a = 0; a < 3; ++a) {
    int e1, e2, ea, sa, goff;
    ghost_face(a, ex, ey, ez, &e1, &e2, &ea, &sa, &goff);
    const double* Gp = gbuf + 36 * voff[p] + goff;
    const int nl = e1 * e2;
    const int nbp = min(ea, NG);  // points of a line within FDP of either end
    // thread per (line, boundary point); the terms of each point in a fixed
    // order, the axes one after the other
    for (int e = threadIdx.x; e < nl * nbp; e += blockDim.x) {
      const int line = e / nbp, idx = e % nbp;
      const int ta = ea <= NG ? idx : (idx < SEA_FDP ? idx : ea - NG + idx);
      const int u1 = line % e1, u2 = line / e1;
      int bx = 0, by = 0, bz = 0;
      if (a == 0) { by = u1; bz = u2; }
      else if (a == 1) { bx = u1; bz = u2; }
      else { bx = u1; by = u2; }
      const int base = (bz * ey + by) * ex + bx;
      // ghost value d below: entry d - 1; above: entry FDP + d - 1
      if (DFM) {
        const DF* G = reinterpret_cast<const DF*>(Gp) + (size_t)line * NG;
        DF add{0.f, 0.f};
#pragma unroll
        for (int k = 1; k <= SEA_FDP; ++k) {
          const DF w{Wd.hi[a][k], Wd.lo[a][k]};
          if (ta - k < 0) add = df_add(add, df_mul(w, G[k - ta - 1]));
          if (ta + k > ea - 1) add = df_add(add, df_mul(w, G[SEA_FDP + ta + k - (ea - 1) - 1]));
        }
        b[base + ta * sa] += df_to_double(add);
      } else {
        const double* G = Gp + (size_t)line * NG;
        double add = 0.0;
#pragma unroll
        for (int k = 1; k <= SEA_FDP; ++k) {
          if (ta - k < 0) add += W.rhs[a][k] * G[k - ta - 1];
          if (ta + k > ea - 1) add += W.rhs[a][k] * G[SEA_FDP + ta + k - (ea - 1) - 1];
        }
        b[base + ta * sa] += add;
      }
    }
    __syncthreads();
  }
}

// Contribution of one axis to q = -Lap_h p at box point t (coordinate u
// along that axis, extent e, stride st), zero outside the box.
__device__ __forceinline__ double lap_axis(const double* __restrict__ pv, int t, int u, int e,
                                           int st, const double* __restrict__ w) {
  double a = 0.0;
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const double L = (u - k >= 0) ? pv[t - k * st] : 0.0;
    const double R = (u + k < e) ? pv[t + k * st] : 0.0;
    a = fma(w[k], L, a);
    a = fma(w[k], R, a);
  }
  return a;
}

// q = -Lap_h p at box point t = (x, y, z): three independent FMA chains
// (one per axis) to keep the FP64 pipe fed.
__device__ __forceinline__ double neg_lap(const double* __restrict__ pv, int t, int x, int y,
                                          int z, int ex, int ey, int ez, const StencilW& W) {
  const double ax = lap_axis(pv, t, x, ex, 1, W.ax[0]);
  const double ay = lap_axis(pv, t, y, ey, ex, W.ax[1]);
  const double az = fma(W.center, pv[t], lap_axis(pv, t, z, ez, ex * ey, W.ax[2]));
  return (ax + ay) + az;
}

// The same operator in double-float on a double-float vector (the mixed
// form's true residual, when the requested tolerance lies well above its
// rounding floor): the FP32 pipes instead of the FP64 unit.
struct StencilOpDF {
  DF ax[3][SEA_FDP + 1];
  DF center;
};
__device__ __forceinline__ DF lap_axis_df(const float2* __restrict__ pv, int t, int u, int e, int st,
                                          const DF* __restrict__ w) {
  DF a{0.f, 0.f};
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const float2 L = (u - k >= 0) ? pv[t - k * st] : make_float2(0.f, 0.f);
    const float2 R = (u + k < e) ? pv[t + k * st] : make_float2(0.f, 0.f);
    a = df_fma(w[k], df_add(DF{L.x, L.y}, DF{R.x, R.y}), a);
  }
  return a;
}
__device__ __forceinline__ DF neg_lap_df(const float2* __restrict__ pv, int t, int x, int y, int z,
                                         int ex, int ey, int ez, const StencilOpDF& W) {
  const DF ax = lap_axis_df(pv, t, x, ex, 1, W.ax[0]);
  const DF ay = lap_axis_df(pv, t, y, ey, ex, W.ax[1]);
  const float2 c = pv[t];
  const DF az = df_fma(W.center, DF{c.x, c.y}, lap_axis_df(pv, t, z, ez, ex * ey, W.ax[2]));
  return df_add(df_add(ax, ay), az);
}

// Walks the points t = t0, t0 + S, t0 + 2S, ... of an ex x ey x ez box in
// [z][y][x] order with their coordinates, without divisions in the loop.
struct BoxWalk {
  int t, x, y, z, dx, dy, dz, ex, ey;
  __device__ BoxWalk(int t0, int S, int ex_, int ey_) : ex(ex_), ey(ey_) {
    t = t0;
    x = t0 % ex;
    y = (t0 / ex) % ey;
    z = t0 / (ex * ey);
    dx = S % ex;
    dy = (S / ex) % ey;
    dz = S / (ex * ey);
  }
  __device__ __forceinline__ void next(int S) {
    t += S;
    x += dx;
    int cy = 0;
    if (x >= ex) {
      x -= ex;
      cy = 1;
    }
    y += dy + cy;
    int cz = 0;
    if (y >= ey) {
      y -= ey;
      cz = 1;
    }
    z += dz + cz;
  }
};

struct CgArgs {
  const double* phi;
  int nx, ny, nz;
  const PairInfo* pinfo;
  const long long* voff;
  const int* order;
  int P;
  double dV, tol;
  int tol_mode, max_iter;
  double *x, *b, *r, *p, *q;
  double* epair;
  int* iters;
  unsigned* status;
  int* queue;
  int warm;  // x holds an initial guess (else the solve starts from 0)
  unsigned long long budget_ns;  // time budget of the launch (0: none)
};

// One pair's FP64 CG (the whole CTA), results into A's per-pair arrays.
__device__ __forceinline__ void cg_pair_fp64(const CgArgs& A, const StencilW& W, int pidx,
                                             double (*red)[32]) {
  const size_t ng = (size_t)A.nx * A.ny * A.nz;
  const PairInfo P = A.pinfo[pidx];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2], n = P.n;
  const long long off = A.voff[pidx];
  double* x = A.x + off;
  const double* b = A.b + off;
  double* r = A.r + off;
  double* pv = A.p + off;
  double* q = A.q + off;

  double rr = 0.0, bb = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double bt = b[t];
    double rt = bt;
    if (A.warm)  // r = b - A x0
      rt = bt - neg_lap(x, t, t % ex, (t / ex) % ey, t / (ex * ey), ex, ey, ez, W);
    r[t] = rt;
    pv[t] = rt;
    rr = fma(rt, rt, rr);
    bb = fma(bt, bt, bb);
  }
  if (!A.warm)
    for (int t = threadIdx.x; t < n; t += blockDim.x) x[t] = 0.0;
  rr = block_sum(rr, red[0]);
  bb = block_sum(bb, red[1]);
  __syncthreads();  // both slot arrays are read before their next use
  const double bnorm = sqrt(bb);
  const double target =
      A.tol_mode == 0 ? A.tol * bnorm : A.tol * 4.0 * 3.14159265358979323846 * sqrt((double)n);
  int it = 0;
  bool done = sqrt(rr) <= target;
  while (!done && it < A.max_iter) {
    double pq = 0.0, pq2 = 0.0;
    {
      const int S = blockDim.x;
      BoxWalk w0(threadIdx.x, 2 * S, ex, ey);
      BoxWalk w1(threadIdx.x + S, 2 * S, ex, ey);
      for (; w1.t < n; w0.next(2 * S), w1.next(2 * S)) {
        const double q0 = neg_lap(pv, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, W);
        const double q1 = neg_lap(pv, w1.t, w1.x, w1.y, w1.z, ex, ey, ez, W);
        q[w0.t] = q0;
        q[w1.t] = q1;
        pq = fma(pv[w0.t], q0, pq);
        pq2 = fma(pv[w1.t], q1, pq2);
      }
      if (w0.t < n) {
        const double q0 = neg_lap(pv, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, W);
        q[w0.t] = q0;
        pq = fma(pv[w0.t], q0, pq);
      }
    }
    pq = block_sum(pq + pq2, red[1]);
    const double alpha = rr / pq;
    double rn = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double pt = pv[t];
      x[t] = fma(alpha, pt, x[t]);
      const double rt = fma(-alpha, q[t], r[t]);
      r[t] = rt;
      rn = fma(rt, rt, rn);
    }
    rn = block_sum(rn, red[0]);
    ++it;
    if (sqrt(rn) <= target) {
      rr = rn;
      done = true;
      break;
    }
    const double beta = rn / rr;
    rr = rn;
    for (int t = threadIdx.x; t < n; t += blockDim.x) pv[t] = fma(beta, pv[t], r[t]);
    __syncthreads();
  }
  // pair integral of Eq. exxGen_mlwf over Omega_ij (skipped for a bare
  // batch of boxes, phi == nullptr)
  const double* fi = A.phi ? A.phi + (size_t)P.i * ng : nullptr;
  const double* fj = A.phi ? A.phi + (size_t)P.j * ng : nullptr;
  double e = 0.0;
  for (int t = threadIdx.x; fi && t < n; t += blockDim.x) {
    const int xx = t % ex, yy = (t / ex) % ey, zz = t / (ex * ey);
    const size_t g = ((size_t)wrapi(P.lo[2] + zz, A.nz) * A.ny + wrapi(P.lo[1] + yy, A.ny)) * A.nx +
                     wrapi(P.lo[0] + xx, A.nx);
    e = fma(fi[g] * fj[g], x[t], e);
  }
  e = block_sum(e, red[1]);
  if (threadIdx.x == 0) {
    if (A.epair) A.epair[pidx] = e * A.dV;
    A.iters[pidx] = done ? it : -it;
    if (!done) atomicOr(A.status, SEA_FLAG_CG_CAP);
  }
}

// The device's nanosecond clock (the same on every SM).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Next queue item for the CTA (thread 0).  With a time budget, once more
// than budget_ns have passed since the CTA started (t0) no further pair is
// taken: the status gets SEA_FLAG_TIMEOUT and the returned item ends the
// CTA's loop (the pairs not taken keep no solution).
__device__ __forceinline__ int claim_item(int* queue, int P, unsigned long long budget_ns,
                                          unsigned long long t0, unsigned* status) {
  if (budget_ns && global_ns() - t0 > budget_ns) {
    atomicOr(status, SEA_FLAG_TIMEOUT);
    return P;
  }
  return atomicAdd(queue, 1);
}

// 3 CTAs per SM: fewer pairs start at once and the longest-first queue
// balances the tail (measured faster than the 4 CTAs/SM the compiler picks).
__global__ void __launch_bounds__(256, 3) k_cg(CgArgs A, StencilW W) {
  __shared__ double red[2][32];
  __shared__ int s_item;
  const unsigned long long t0 = A.budget_ns ? global_ns() : 0ull;
  for (;;) {
    if (threadIdx.x == 0) s_item = claim_item(A.queue, A.P, A.budget_ns, t0, A.status);
    __syncthreads();
    const int item = s_item;
    if (item >= A.P) break;
    const int pidx = A.order[item];
    cg_pair_fp64(A, W, pidx, red);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision form: FP32 stencil sweeps and CG vectors, FP64 where the
// accuracy is decided.  Per pair, iterative refinement:
//   x = 0 (FP64), r = b (FP64)
//   while ||r||_2 > tol ||b||_2 (FP64 norm of the true FP64 residual):
//     solve A d = r / ||r|| by CG in FP32 to a relative residual of
//       SEA_MIXED_INNER (dot products: per-thread partial sums in
//       compensated FP32 -- exact products by FMA, error-free additions --
//       combined across the block by error-free FP32 additions; alpha,
//       beta and the inner stopping test in FP32: on this part one FP64
//       instruction of a warp costs the time of 64 FP32 ones, and the
//       inner solve needs only SEA_MIXED_INNER)
//     x += ||r|| d (FP64);  r = b - A x (FP64 stencil)
// The stopping rule is applied to the true FP64 residual, so the result
// meets the same bound as the FP64 solver.
// ---------------------------------------------------------------------------
#define SEA_MIXED_INNER 1e-4f
// CTA size of the mixed CG (one pair per CTA at a time)
#define SEA_CG_THREADS 512
#define SEA_MIXED_MAX_OUTER 30
// smallest relative tolerance for which the true residual is formed in
// double-float (below it, in FP64)
#define SEA_DF_RESIDUAL_TOL 1e-10

struct StencilWf {
  float ax[3][SEA_FDP + 1];
  float center;
};

// Compensated FP32 accumulator of a sum of products (value = hi + lo).
struct DotF {
  float hi, lo;
  __device__ DotF() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // exact product = p + pe
    const float s = hi + p;
    const float bb = s - hi;
    const float se = (hi - (s - bb)) + (p - bb);  // exact sum = s + se
    hi = s;
    lo += se + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// (hi, lo) += (bh, bl) with an error-free addition of the leading parts.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float v = s - hi;
  const float e = (hi - (s - v)) + (bh - v);
  hi = s;
  lo = (lo + bl) + e;
}

// Block sum of compensated (hi, lo) partials in FP32 only: warp butterfly,
// then every warp combines the warps' results by a second butterfly (the
// error-free addition is symmetric in its operands, so every lane ends with
// the same bits).  `slots` holds 32 float2 of shared memory, reused only
// after the next __syncthreads.  Returns hi + lo rounded to FP32 (the same
// value in every thread).
__device__ __forceinline__ float block_sum_f(float hi, float lo, float2* slots) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    two_sum_add(hi, lo, bh, bl);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) slots[w] = make_float2(hi, lo);
  __syncthreads();
  const float2 t = lane < nw ? slots[lane] : make_float2(0.f, 0.f);
  hi = t.x;
  lo = t.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    two_sum_add(hi, lo, bh, bl);
  }
  return hi + lo;
}

__device__ __forceinline__ float lap_axis_f(const float* __restrict__ pv, int t, int u, int e,
                                            int st, const float* __restrict__ w) {
  float a = 0.f;
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const float L = (u - k >= 0) ? pv[t - k * st] : 0.f;
    const float R = (u + k < e) ? pv[t + k * st] : 0.f;
    a = fmaf(w[k], L, a);
    a = fmaf(w[k], R, a);
  }
  return a;
}

__device__ __forceinline__ float neg_lap_f(const float* __restrict__ pv, int t, int x, int y,
                                           int z, int ex, int ey, int ez, const StencilWf& W) {
  const float ax = lap_axis_f(pv, t, x, ex, 1, W.ax[0]);
  const float ay = lap_axis_f(pv, t, y, ey, ex, W.ax[1]);
  const float az = fmaf(W.center, pv[t], lap_axis_f(pv, t, z, ez, ex * ey, W.ax[2]));
  return (ax + ay) + az;
}

// Shared-memory layout of the mixed CG's residual: the pair box's planes of
// ex x ey points stored row after row (so consecutive points of a warp sit
// in consecutive banks), each plane followed by F = SEA_FDP zero rows, which
// serve as the y halo on both sides, and F zero planes before and after the
// box for the z halo.  Box point t = (z ey + y) ex + x sits at
// org + t + z F ex.  Neighbours along y and z outside the box read zeros;
// along x they are masked.
__host__ __device__ __forceinline__ int cg_pad_volume(int ex, int ey, int ez) {
  return ex * (ey + SEA_FDP) * (ez + 2 * SEA_FDP);
}

// -Lap_h r at padded index tp (box x coordinate x, row length ex, plane
// size PXY): the same products and order as neg_lap_f.
__device__ __forceinline__ float neg_lap_pad(const float* __restrict__ pv, int tp, int x, int ex,
                                             int PXY, const StencilWf& W) {
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const float L = pv[tp - k], R = pv[tp + k];
    ax = fmaf(W.ax[0][k], x - k >= 0 ? L : 0.f, ax);
    ax = fmaf(W.ax[0][k], x + k < ex ? R : 0.f, ax);
  }
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    ay = fmaf(W.ax[1][k], pv[tp - k * ex], ay);
    ay = fmaf(W.ax[1][k], pv[tp + k * ex], ay);
  }
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    az = fmaf(W.ax[2][k], pv[tp - k * PXY], az);
    az = fmaf(W.ax[2][k], pv[tp + k * PXY], az);
  }
  az = fmaf(W.center, pv[tp], az);
  return (ax + ay) + az;
}

// Block sum of two FP32 values at once (one barrier): warp butterfly, then
// every warp combines the warps' results by a second butterfly, so every
// thread gets the same bits.  `slots` holds 32 float2 of shared memory,
// reused only after the next __syncthreads.
__device__ __forceinline__ float2 block_sum2_f(float a, float b, float2* slots) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) slots[w] = make_float2(a, b);
  __syncthreads();
  float2 t = lane < nw ? slots[lane] : make_float2(0.f, 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
  }
  return t;
}

// Inner solve in the single-reduction arrangement of CG (Chronopoulos and
// Gear, 1989): per iteration one stencil product w = A r and one block
// reduction of (r, r) and (w, r), then
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old)
//   p = r + beta p,  s = w + beta s,  d += alpha p,  r -= alpha s
// (beta = 0, alpha = gamma / delta at the first step), which is CG in exact
// arithmetic with two barriers per iteration instead of four.  The residual r
// lives in shared memory in the padded layout above (no bounds tests along
// y and z, consecutive points in consecutive banks); p, s, w and d in global
// memory (L1-resident).  Stops when
// (r, r) <= SEA_MIXED_INNER^2 (r0, r0).  For pairs whose padded box fits the
// shared buffer.  Ends with x += rnorm d (FP64).  Returns the new total of
// inner iterations (stencil products followed by an update).
template <bool DRES>
__device__ __forceinline__ int inner_cg_smem(const double* __restrict__ r, double rnorm,
                                             double* __restrict__ x, float* __restrict__ d,
                                             float* __restrict__ pf, float* __restrict__ sf,
                                             float* __restrict__ wf, float* __restrict__ rS,
                                             int n, int ex, int ey, int ez, const StencilWf& Wf,
                                             float2* fs0, float2* fs1, int inner_total,
                                             int max_iter) {
  const int S = blockDim.x;
  const int PXY = ex * (ey + SEA_FDP), gap = SEA_FDP * ex;
  const int Vp = PXY * (ez + 2 * SEA_FDP);
  const int org = SEA_FDP * PXY;  // padded index of box point (0, 0, 0)
  for (int t = threadIdx.x; t < Vp; t += S) rS[t] = 0.f;
  __syncthreads();
  const double inv = 1.0 / rnorm;
  const float invf = (float)inv;
  {
    BoxWalk w(threadIdx.x, S, ex, ey);
    for (; w.t < n; w.next(S)) {
      if (DRES) {
        const float2 rv = reinterpret_cast<const float2*>(r)[w.t];
        rS[org + w.t + w.z * gap] = fmaf(rv.x, invf, rv.y * invf);
      } else {
        rS[org + w.t + w.z * gap] = (float)(r[w.t] * inv);
      }
      pf[w.t] = 0.f;
      sf[w.t] = 0.f;
      d[w.t] = 0.f;
    }
  }
  __syncthreads();
  float stop = 0.f, gamma_old = 1.f, alpha_old = 1.f;
  float2* slots[2] = {fs0, fs1};
  for (int it = 0;; ++it) {
    float g = 0.f, dl = 0.f;
    {
      BoxWalk w(threadIdx.x, S, ex, ey);
      for (; w.t < n; w.next(S)) {
        const int tp = org + w.t + w.z * gap;
        const float wv = neg_lap_pad(rS, tp, w.x, ex, PXY, Wf);
        const float rv = rS[tp];
        wf[w.t] = wv;
        g = fmaf(rv, rv, g);
        dl = fmaf(wv, rv, dl);
      }
    }
    const float2 gd = block_sum2_f(g, dl, slots[it & 1]);
    const float gamma = gd.x, delta = gd.y;
    if (it == 0) stop = (float)SEA_MIXED_INNER * (float)SEA_MIXED_INNER * gamma;
    if (gamma <= stop || inner_total >= max_iter) break;
    const float beta = it == 0 ? 0.f : gamma / gamma_old;
    const float alpha = it == 0 ? gamma / delta : gamma / (delta - beta * gamma / alpha_old);
    {
      BoxWalk w(threadIdx.x, S, ex, ey);
      for (; w.t < n; w.next(S)) {
        const int tp = org + w.t + w.z * gap;
        const float rv = rS[tp];
        const float pv = fmaf(beta, pf[w.t], rv);
        const float sv = fmaf(beta, sf[w.t], wf[w.t]);
        pf[w.t] = pv;
        sf[w.t] = sv;
        d[w.t] = fmaf(alpha, pv, d[w.t]);
        rS[tp] = fmaf(-alpha, sv, rv);
      }
    }
    gamma_old = gamma;
    alpha_old = alpha;
    ++inner_total;
    __syncthreads();
  }
  if (DRES) {
    float2* xd = reinterpret_cast<float2*>(x);
    const DF rn = df_from_double(rnorm);
    for (int t = threadIdx.x; t < n; t += S) {
      const float2 xv = xd[t];
      const DF y = df_add(df_mul_f(d[t], rn), DF{xv.x, xv.y});
      xd[t] = make_float2(y.hi, y.lo);
    }
  } else {
    for (int t = threadIdx.x; t < n; t += S) x[t] = fma(rnorm, (double)d[t], x[t]);
  }
  __syncthreads();  // rS is free for the next pair
  return inner_total;
}

struct CgMixedArgs {
  const double* phi;
  int nx, ny, nz;
  const PairInfo* pinfo;
  const long long* voff;
  const int* order;
  int P;
  double dV, tol;
  int tol_mode, max_iter;
  double *x, *b, *r;       // FP64: solution, right-hand side, true residual
  float *d, *rf, *pf, *qf;  // FP32 inner-solve vectors
  double* epair;
  int* iters;     // total inner iterations (negative if capped)
  int* outers;    // refinement steps
  unsigned* status;
  int* queue;
  int warm;       // x holds an initial guess (else the solve starts from 0)
  int pad_cap;    // floats of shared memory for the padded search direction
  unsigned long long budget_ns;  // time budget of the launch (0: none)
};

// block_sum with the serial combine done by one warp (the same order, so the
// same bits) and the total broadcast through *bc: an FP64 instruction costs
// a warp the same time however many of its lanes are active, so the warps of
// a large CTA should not all repeat the combine.
__device__ __forceinline__ double block_sum_1w(double v, double* slots, double* bc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) slots[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += slots[k];
    if (threadIdx.x == 0) *bc = s;
  }
  __syncthreads();
  return *bc;
}

// One pair's mixed-precision solve (the whole CTA).
__device__ __forceinline__ void cg_pair_mixed(const CgMixedArgs& A, const StencilW& W,
                                              const StencilWf& Wf, int pidx, double (*red)[32],
                                              double* bc, float* pS) {
  const size_t ng = (size_t)A.nx * A.ny * A.nz;
  const int S = blockDim.x;
  const PairInfo P = A.pinfo[pidx];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2], n = P.n;
  const long long off = A.voff[pidx];
  double* x = A.x + off;
  const double* b = A.b + off;
  double* r = A.r + off;
  float* d = A.d + off;
  float* rf = A.rf + off;
  float* pf = A.pf + off;
  float* qf = A.qf + off;

  // The true residual in double-float (x and r held as FP32 pairs in their
  // FP64 arrays until the end) when the tolerance is at least
  // SEA_DF_RESIDUAL_TOL: its rounding floor, about 2^-47 of the stencil's
  // largest terms (a few 10^-12 of ||b||), then stays far below the target.
  const bool dres = A.tol_mode == 0 && A.tol >= SEA_DF_RESIDUAL_TOL;
  __shared__ StencilOpDF Wo;
  float2* xd = reinterpret_cast<float2*>(x);
  float2* rd = reinterpret_cast<float2*>(r);
  double bb = 0.0, rr0 = 0.0;
  if (dres) {
    if (threadIdx.x < 3 * (SEA_FDP + 1))
      Wo.ax[threadIdx.x / (SEA_FDP + 1)][threadIdx.x % (SEA_FDP + 1)] =
          df_from_double(W.ax[threadIdx.x / (SEA_FDP + 1)][threadIdx.x % (SEA_FDP + 1)]);
    if (threadIdx.x == 3 * (SEA_FDP + 1)) Wo.center = df_from_double(W.center);
    for (int t = threadIdx.x; t < n; t += S) {
      const float2 xv = A.warm ? split64(x[t]) : make_float2(0.f, 0.f);
      xd[t] = xv;
    }
    __syncthreads();
    float rr0f = 0.f;
    BoxWalk w(threadIdx.x, S, ex, ey);
    for (; w.t < n; w.next(S)) {
      const double bt = b[w.t];
      const float2 bs = split64(bt);
      DF rt{bs.x, bs.y};
      if (A.warm) rt = df_add(rt, df_neg(neg_lap_df(xd, w.t, w.x, w.y, w.z, ex, ey, ez, Wo)));
      rd[w.t] = make_float2(rt.hi, rt.lo);
      bb = fma(bt, bt, bb);
      rr0f = fmaf(rt.hi, rt.hi, rr0f);
    }
    rr0 = (double)rr0f;
  } else {
    for (int t = threadIdx.x; t < n; t += S) {
      const double bt = b[t];
      double rt = bt;
      if (A.warm)  // r = b - A x0
        rt = bt - neg_lap(x, t, t % ex, (t / ex) % ey, t / (ex * ey), ex, ey, ez, W);
      r[t] = rt;
      bb = fma(bt, bt, bb);
      rr0 = fma(rt, rt, rr0);
    }
    if (!A.warm)
      for (int t = threadIdx.x; t < n; t += S) x[t] = 0.0;
  }
  bb = block_sum_1w(bb, red[0], bc);
  rr0 = block_sum_1w(rr0, red[1], bc);
  __syncthreads();  // both slot arrays are read before their next use
  const double bnorm = sqrt(bb);
  const double target =
      A.tol_mode == 0 ? A.tol * bnorm : A.tol * 4.0 * 3.14159265358979323846 * sqrt((double)n);
  double rnorm = sqrt(rr0);
  int inner_total = 0, outer = 0;
  bool done = rnorm <= target, capped = false;
  while (!done) {
    if (outer >= SEA_MIXED_MAX_OUTER || inner_total >= A.max_iter) {
      capped = true;
      break;
    }
    // inner FP32 CG on A d = r / ||r||: vectors, scalars and the block
    // reductions (compensated partials) all in FP32
    float2* fs0 = reinterpret_cast<float2*>(red[0]);
    float2* fs1 = reinterpret_cast<float2*>(red[1]);
    if (cg_pad_volume(ex, ey, ez) <= A.pad_cap) {
      inner_total = dres ? inner_cg_smem<true>(r, rnorm, x, d, pf, rf, qf, pS, n, ex, ey, ez, Wf,
                                               fs0, fs1, inner_total, A.max_iter)
                         : inner_cg_smem<false>(r, rnorm, x, d, pf, rf, qf, pS, n, ex, ey, ez, Wf,
                                                fs0, fs1, inner_total, A.max_iter);
    } else {
    const double inv = 1.0 / rnorm;
    DotF rr0;
    for (int t = threadIdx.x; t < n; t += S) {
      const float v = dres ? fmaf(rd[t].x, (float)inv, rd[t].y * (float)inv) : (float)(r[t] * inv);
      rf[t] = v;
      pf[t] = v;
      d[t] = 0.f;
      rr0.add(v, v);
    }
    float rr = block_sum_f(rr0.hi, rr0.lo, fs1);
    const float stop = (float)SEA_MIXED_INNER * (float)SEA_MIXED_INNER * rr;  // on ||r||^2
    while (rr > stop && inner_total < A.max_iter) {
      DotF pq0, pq1;
      {
        BoxWalk w0(threadIdx.x, 2 * S, ex, ey);
        BoxWalk w1(threadIdx.x + S, 2 * S, ex, ey);
        for (; w1.t < n; w0.next(2 * S), w1.next(2 * S)) {
          const float q0 = neg_lap_f(pf, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, Wf);
          const float q1 = neg_lap_f(pf, w1.t, w1.x, w1.y, w1.z, ex, ey, ez, Wf);
          qf[w0.t] = q0;
          qf[w1.t] = q1;
          pq0.add(pf[w0.t], q0);
          pq1.add(pf[w1.t], q1);
        }
        if (w0.t < n) {
          const float q0 = neg_lap_f(pf, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, Wf);
          qf[w0.t] = q0;
          pq0.add(pf[w0.t], q0);
        }
      }
      two_sum_add(pq0.hi, pq0.lo, pq1.hi, pq1.lo);
      const float pq = block_sum_f(pq0.hi, pq0.lo, fs0);
      const float alpha = rr / pq;
      DotF rn0;
      for (int t = threadIdx.x; t < n; t += S) {
        d[t] = fmaf(alpha, pf[t], d[t]);
        const float rt = fmaf(-alpha, qf[t], rf[t]);
        rf[t] = rt;
        rn0.add(rt, rt);
      }
      const float rn = block_sum_f(rn0.hi, rn0.lo, fs1);
      ++inner_total;
      const float beta = rn / rr;
      rr = rn;
      if (rn <= stop) break;
      for (int t = threadIdx.x; t < n; t += S) pf[t] = fmaf(beta, pf[t], rf[t]);
      __syncthreads();
    }
    // correction of x (FP64, or double-float with dres)
    if (dres) {
      const DF rn = df_from_double(rnorm);
      for (int t = threadIdx.x; t < n; t += S) {
        const DF y = df_add(df_mul_f(d[t], rn), DF{xd[t].x, xd[t].y});
        xd[t] = make_float2(y.hi, y.lo);
      }
    } else {
      for (int t = threadIdx.x; t < n; t += S) x[t] = fma(rnorm, (double)d[t], x[t]);
    }
    }
    __syncthreads();
    // true residual
    double r2 = 0.0;
    if (dres) {
      float r2f = 0.f;
      BoxWalk w0(threadIdx.x, S, ex, ey);
      for (; w0.t < n; w0.next(S)) {
        const float2 bs = split64(b[w0.t]);
        const DF rt = df_add(DF{bs.x, bs.y},
                             df_neg(neg_lap_df(xd, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, Wo)));
        rd[w0.t] = make_float2(rt.hi, rt.lo);
        r2f = fmaf(rt.hi, rt.hi, r2f);
      }
      r2 = (double)r2f;
    } else {
      BoxWalk w0(threadIdx.x, S, ex, ey);
      for (; w0.t < n; w0.next(S)) {
        const double rt = b[w0.t] - neg_lap(x, w0.t, w0.x, w0.y, w0.z, ex, ey, ez, W);
        r[w0.t] = rt;
        r2 = fma(rt, rt, r2);
      }
    }
    rnorm = sqrt(block_sum_1w(r2, red[0], bc));
    ++outer;
    done = rnorm <= target;
  }
  if (dres) {  // x back to FP64 (each thread converts the points it wrote)
    for (int t = threadIdx.x; t < n; t += S) {
      const float2 xv = xd[t];
      x[t] = df_to_double(DF{xv.x, xv.y});
    }
    __syncthreads();
  }
  // pair integral of Eq. exxGen_mlwf over Omega_ij
  const double* fi = A.phi ? A.phi + (size_t)P.i * ng : nullptr;
  const double* fj = A.phi ? A.phi + (size_t)P.j * ng : nullptr;
  double e = 0.0;
  for (int t = threadIdx.x; fi && t < n; t += S) {
    const int xx = t % ex, yy = (t / ex) % ey, zz = t / (ex * ey);
    const size_t g = ((size_t)wrapi(P.lo[2] + zz, A.nz) * A.ny + wrapi(P.lo[1] + yy, A.ny)) * A.nx +
                     wrapi(P.lo[0] + xx, A.nx);
    e = fma(fi[g] * fj[g], x[t], e);
  }
  e = block_sum_1w(e, red[1], bc);
  if (threadIdx.x == 0) {
    if (A.epair) A.epair[pidx] = e * A.dV;
    A.iters[pidx] = capped ? -inner_total : inner_total;
    if (A.outers) A.outers[pidx] = outer;
    if (capped) atomicOr(A.status, SEA_FLAG_CG_CAP);
  }
}

__global__ void __launch_bounds__(SEA_CG_THREADS, 1024 / SEA_CG_THREADS) k_cg_mixed(CgMixedArgs A, StencilW W, StencilWf Wf) {
  __shared__ double red[2][32];
  __shared__ int s_item;
  __shared__ double bc;
  extern __shared__ float pS[];  // A.pad_cap floats
  const unsigned long long t0 = A.budget_ns ? global_ns() : 0ull;
  for (;;) {
    if (threadIdx.x == 0) s_item = claim_item(A.queue, A.P, A.budget_ns, t0, A.status);
    __syncthreads();
    const int item = s_item;
    if (item >= A.P) break;
    const int pidx = A.order[item];
    cg_pair_mixed(A, W, Wf, pidx, red, &bc, pS);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Batched form: the pairs of several independent configurations in one
// persistent launch.  items[k] = (configuration, rank): the pair of that
// rank in the configuration's longest-first order; the item list deals the
// ranks round-robin over the configurations, so the longest pairs of every
// configuration start first.  Each configuration brings its own grid,
// stencil weights and buffers.
// ---------------------------------------------------------------------------
struct BatchCg {
  CgArgs a;
  CgMixedArgs m;
  StencilW W;
  StencilWf Wf;
  int mixed;
};

// MIXED: the items are all mixed-form (CTA of SEA_CG_THREADS, as k_cg_mixed)
// or all FP64 (CTA of 256, as k_cg), so every pair is solved with the same
// CTA size, hence the same bits, as in its own configuration's launch.
template <bool MIXED>
__global__ void __launch_bounds__(MIXED ? SEA_CG_THREADS : 256, MIXED ? 1024 / SEA_CG_THREADS : 2)
    k_cg_batch(const BatchCg* __restrict__ descs, const int2* __restrict__ items, int total,
               int* __restrict__ queue) {
  __shared__ double red[2][32];
  __shared__ int s_item;
  __shared__ BatchCg d;
  __shared__ double bc;
  extern __shared__ float pS[];  // the largest pad_cap of the descriptors
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int2 it = items[item];
    {
      const int* src = (const int*)(descs + it.x);
      int* dst = (int*)&d;
      for (int w = threadIdx.x; w < (int)(sizeof(BatchCg) / sizeof(int)); w += blockDim.x)
        dst[w] = src[w];
    }
    __syncthreads();
    if (MIXED)
      cg_pair_mixed(d.m, d.W, d.Wf, d.m.order[it.y], red, &bc, pS);
    else
      cg_pair_fp64(d.a, d.W, d.a.order[it.y], red);
    __syncthreads();
  }
}

static StencilW make_weights(const sea_ctx* c) {
  StencilW W;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= SEA_FDP; ++k) {
      W.ax[a][k] = c->w_ax[a][k];
      W.rhs[a][k] = -c->w_ax[a][k];
    }
  W.center = c->w_center;
  return W;
}

cudaError_t launch_pair_setup(sea_ctx* c) {
  if (c->P == 0) return cudaSuccess;
  auto moments = c->prm.precision == 1 ? k_pair_moments<true> : k_pair_moments<false>;
  const size_t msm = pair_moments_smem(c->N[1], c->N[2]);
  if (msm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)msm);
    if (e != cudaSuccess) return e;
  }
  moments<<<c->P, 256, msm, c->stream>>>(
      (const double*)c->phi.p, c->N[0], c->N[1], c->N[2], (const PairInfo*)c->pinfo.p,
      (const long long*)c->voff.p, c->h[0], c->h[1], c->h[2], c->dV, c->prm.lmax,
      (double*)c->bbuf.p, (double*)c->Q.p, (const int*)c->order.p);
  if (!sea_ensure(c, c->gbuf, (size_t)36 * std::max<long long>(c->U, 1) * sizeof(double)))
    return cudaErrorMemoryAllocation;
  auto geval = c->prm.precision == 1 ? k_ghost_eval<true> : k_ghost_eval<false>;
  auto gapply = c->prm.precision == 1 ? k_boundary_apply<true> : k_boundary_apply<false>;
  const StencilW W = make_weights(c);
  StencilWd Wd;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= SEA_FDP; ++k) {
      Wd.hi[a][k] = (float)W.rhs[a][k];
      Wd.lo[a][k] = (float)(W.rhs[a][k] - (double)Wd.hi[a][k]);
    }
  geval<<<dim3(3, c->P), 256, 0, c->stream>>>(
      (const PairInfo*)c->pinfo.p, (const long long*)c->voff.p, c->h[0], c->h[1], c->h[2],
      (const double*)c->Q.p, (double*)c->gbuf.p, (const int*)c->order.p);
  gapply<<<c->P, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p, (const long long*)c->voff.p, W,
                                      Wd, (const double*)c->gbuf.p, (double*)c->bbuf.p,
                                      (const int*)c->order.p);
  c->launches += 3;
  return cudaGetLastError();
}

static StencilWf make_weights_f(const StencilW& W) {
  StencilWf F;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k <= SEA_FDP; ++k) F.ax[a][k] = (float)W.ax[a][k];
  F.center = (float)W.center;
  return F;
}

static CgMixedArgs mixed_args(sea_ctx* c) {
  CgMixedArgs A;
  memset(&A, 0, sizeof(A));
  A.phi = (const double*)c->phi.p;
  A.nx = c->N[0];
  A.ny = c->N[1];
  A.nz = c->N[2];
  A.pinfo = (const PairInfo*)c->pinfo.p;
  A.voff = (const long long*)c->voff.p;
  A.order = (const int*)c->order.p;
  A.P = c->P;
  A.dV = c->dV;
  A.tol = c->prm.cg_tol;
  A.tol_mode = c->prm.cg_tol_mode;
  A.max_iter = c->prm.cg_max_iter;
  A.x = (double*)c->vbuf.p;
  A.b = (double*)c->bbuf.p;
  A.r = (double*)c->rbuf.p;
  // FP32 vectors: two per FP64-sized buffer
  A.d = (float*)c->pbuf.p;
  A.rf = A.d + c->U;
  A.pf = (float*)c->qbuf.p;
  A.qf = A.pf + c->U;
  A.epair = (double*)c->epair.p;
  A.iters = (int*)c->iters.p;
  A.outers = nullptr;
  A.status = (unsigned*)c->status.p;
  A.queue = (int*)c->queue.p;
  A.pad_cap = cg_pad_cap(c);
  A.warm = c->cg_warm ? 1 : 0;
  A.budget_ns = (unsigned long long)(c->prm.timeout_ms * 1e6);
  return A;
}

static CgArgs fp64_args(sea_ctx* c) {
  CgArgs A;
  memset(&A, 0, sizeof(A));
  A.phi = (const double*)c->phi.p;
  A.nx = c->N[0];
  A.ny = c->N[1];
  A.nz = c->N[2];
  A.pinfo = (const PairInfo*)c->pinfo.p;
  A.voff = (const long long*)c->voff.p;
  A.order = (const int*)c->order.p;
  A.P = c->P;
  A.dV = c->dV;
  A.tol = c->prm.cg_tol;
  A.tol_mode = c->prm.cg_tol_mode;
  A.max_iter = c->prm.cg_max_iter;
  A.x = (double*)c->vbuf.p;
  A.b = (double*)c->bbuf.p;
  A.r = (double*)c->rbuf.p;
  A.p = (double*)c->pbuf.p;
  A.q = (double*)c->qbuf.p;
  A.epair = (double*)c->epair.p;
  A.iters = (int*)c->iters.p;
  A.status = (unsigned*)c->status.p;
  A.queue = (int*)c->queue.p;
  A.warm = c->cg_warm ? 1 : 0;
  A.budget_ns = (unsigned long long)(c->prm.timeout_ms * 1e6);
  return A;
}

// Shared memory of the mixed CG's padded search direction: the largest
// padded pair box, at most SEA_CG_PAD_LIMIT floats (four CTAs per SM);
// pairs above the limit solve on global vectors.
#define SEA_CG_PAD_LIMIT 13824
int cg_pad_cap(const sea_ctx* c) {
  return c->prm.precision == 1 ? std::min(c->cg_pad_max, SEA_CG_PAD_LIMIT) : 0;
}

cudaError_t launch_cg(sea_ctx* c) {
  if (c->P == 0) return cudaSuccess;
  int nsm = 0, occ = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int pad_cap = cg_pad_cap(c);
  const size_t smem = (size_t)pad_cap * sizeof(float);
  if (c->prm.precision == 1) {
    cudaError_t e = cudaFuncSetAttribute(k_cg_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(SEA_CG_PAD_LIMIT * sizeof(float)));
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_mixed, SEA_CG_THREADS, smem);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg, 256, 0);
  }
  if (occ < 1) occ = 1;
  const int grid = min(c->P, nsm * occ);
  cudaMemsetAsync(c->queue.p, 0, sizeof(int), c->stream);
  const StencilW W = make_weights(c);
  if (c->prm.precision == 1)
    k_cg_mixed<<<grid, SEA_CG_THREADS, smem, c->stream>>>(mixed_args(c), W, make_weights_f(W));
  else
    k_cg<<<grid, 256, 0, c->stream>>>(fp64_args(c), W);
  c->launches += 1;
  return cudaGetLastError();
}

// Damped Jacobi sweeps on every pair's starting vector x (CTA per pair):
// x += omega (b - A x) / diag(A).  Removes the high-frequency part of a
// guess's error, which A would otherwise amplify in the CG's first residual.
__global__ void __launch_bounds__(256)
    k_smooth(const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff, int P,
             const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
             StencilW W, int sweeps, double omega) {
  const int p = blockIdx.x;
  if (p >= P) return;
  const PairInfo Pi = pinfo[p];
  const int ex = Pi.ext[0], ey = Pi.ext[1], ez = Pi.ext[2], n = Pi.n;
  const long long off = voff[p];
  const double s = omega / W.center;
  for (int k = 0; k < sweeps; ++k) {
    for (int t = threadIdx.x; t < n; t += blockDim.x)
      r[off + t] = b[off + t] - neg_lap(x + off, t, t % ex, (t / ex) % ey, t / (ex * ey), ex, ey, ez, W);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) x[off + t] = fma(s, r[off + t], x[off + t]);
    __syncthreads();
  }
}

cudaError_t launch_smooth(sea_ctx* c, int sweeps, double omega) {
  if (c->P == 0 || sweeps <= 0) return cudaSuccess;
  k_smooth<<<c->P, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p, (const long long*)c->voff.p,
                                        c->P, (const double*)c->bbuf.p, (double*)c->vbuf.p,
                                        (double*)c->rbuf.p, make_weights(c), sweeps, omega);
  c->launches += 1;
  return cudaGetLastError();
}

// Descriptor of one configuration for k_cg_batch (host side).
void make_batch_desc(sea_ctx* c, void* out) {
  BatchCg d;
  memset(&d, 0, sizeof(d));
  d.a = fp64_args(c);
  d.m = mixed_args(c);
  d.a.budget_ns = d.m.budget_ns = 0;  // the batched launch has no time budget
  d.W = make_weights(c);
  d.Wf = make_weights_f(d.W);
  d.mixed = c->prm.precision == 1;
  memcpy(out, &d, sizeof(d));
}

size_t batch_desc_bytes() { return sizeof(BatchCg); }

int cg_batch_max_ctas_per_sm(int device, int pad_cap, bool mixed) {
  const size_t smem = (size_t)pad_cap * sizeof(float);
  const int threads = mixed ? SEA_CG_THREADS : 256;
  auto kern = mixed ? k_cg_batch<true> : k_cg_batch<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(SEA_CG_PAD_LIMIT * sizeof(float))) != cudaSuccess)
    return 1;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
  (void)device;
  return occ < 1 ? 1 : occ;
}

cudaError_t launch_cg_batch(cudaStream_t st, int device, const void* descs, const int2* items,
                            int total, int* queue, int pad_cap, bool mixed, int ctas_per_sm) {
  if (total == 0) return cudaSuccess;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const size_t smem = (size_t)pad_cap * sizeof(float);
  const int threads = mixed ? SEA_CG_THREADS : 256;
  auto kern = mixed ? k_cg_batch<true> : k_cg_batch<false>;
  const int occ = cg_batch_max_ctas_per_sm(device, pad_cap, mixed);
  const int per_sm = ctas_per_sm >= 1 ? min(ctas_per_sm, occ) : occ;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  kern<<<min(total, nsm * per_sm), threads, smem, st>>>((const BatchCg*)descs, items, total, queue);
  return cudaGetLastError();
}

// Batched solve of -Lap_h x = rhs on independent boxes (no pair energies):
// boxes[] and voff[] on the device, order[] the processing order; r, p, q
// scratch of the same total length as x.
cudaError_t launch_cg_boxes(cudaStream_t stream, int device, const double h[3], int nbox,
                            const PairInfo* boxes, const long long* voff, const int* order,
                            const double* rhs, double* x, double* r, double* p, double* q,
                            int* iters, unsigned* status, int* queue, double tol, int tol_mode,
                            int max_iter) {
  if (nbox == 0) return cudaSuccess;
  double w[SEA_FDP + 1];
  fornberg_weights(w);
  StencilW W;
  W.center = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double ih2 = 1.0 / (h[a] * h[a]);
    for (int k = 0; k <= SEA_FDP; ++k) {
      W.ax[a][k] = -w[k] * ih2;
      W.rhs[a][k] = w[k] * ih2;
    }
    W.center += -w[0] * ih2;
  }
  int nsm = 0, occ = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg, 256, 0);
  if (occ < 1) occ = 1;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  CgArgs A;
  memset(&A, 0, sizeof(A));
  A.phi = nullptr;
  A.nx = A.ny = A.nz = 1;
  A.pinfo = boxes;
  A.voff = voff;
  A.order = order;
  A.P = nbox;
  A.dV = h[0] * h[1] * h[2];
  A.tol = tol;
  A.tol_mode = tol_mode;
  A.max_iter = max_iter;
  A.x = x;
  A.b = (double*)rhs;
  A.r = r;
  A.p = p;
  A.q = q;
  A.epair = nullptr;
  A.iters = iters;
  A.status = status;
  A.queue = queue;
  k_cg<<<min(nbox, nsm * occ), 256, 0, stream>>>(A, W);
  return cudaGetLastError();
}

cudaError_t upload_harmonics_pair() { return upload_harmonics_here(); }

}  // namespace sea
