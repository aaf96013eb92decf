// sea_internal.cuh -- device helpers and the context of the GB300 exx engine.
//
// Everything here belongs to the CUDA library (libsea.so).  It is written
// from the paper's equations; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "../../include/sea.h"

#define SEA_LMAX 6
#define SEA_NQ ((SEA_LMAX + 1) * (SEA_LMAX + 1))
#define SEA_FDP 6  // stencil half width: O(h^12) second difference (App. C)

// Status bits written by kernels (device word, read back by the host).
#define SEA_FLAG_CG_CAP 1u
#define SEA_FLAG_NOT_PD 2u
#define SEA_FLAG_BOUNDS 4u
#define SEA_FLAG_NONFINITE 8u

namespace sea {

__host__ __device__ inline int wrapi(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

__host__ __device__ inline int lmi(int l, int m) { return l * l + l + m; }

// Coefficients of the real solid-harmonic recurrences in Racah
// normalization (C_l0 = r^l P_l(cos theta)), filled by the host:
//   C_{l+1,+-(l+1)} = top[l] (x C_{l,l} -+ y C_{l,-l}),  (x C_00 / y C_00 at l = 0)
//   C_{l+1,m} = mid_b[l][m] z C_{l,m} - mid_c[l][m] r^2 C_{l-1,m},  |m| <= l.
// With Q_lm = sum rho C_lm dV, the multipole potential of Eq. me is
//   v(r) = sum_lm Q_lm C_lm(r) / r^(2l+1)
// (the orthonormal form 4 pi Q Y /((2l+1) r^(l+1)) with the (2l+1)/(4 pi)
// normalization folded into C).
struct HarmCoef {
  double top[SEA_LMAX];
  double mid_b[SEA_LMAX][2 * SEA_LMAX + 1];
  double mid_c[SEA_LMAX][2 * SEA_LMAX + 1];
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

// All regular solid harmonics C_lm(x, y, z), l <= SEA_LMAX.
__device__ __forceinline__ void solid_regular(double x, double y, double z, double* C) {
  const double r2 = x * x + y * y + z * z;
  C[0] = 1.0;
#pragma unroll
  for (int l = 0; l < SEA_LMAX; ++l) {
    const double t = c_harm.top[l];
    if (l == 0) {
      C[lmi(1, 1)] = t * x;
      C[lmi(1, -1)] = t * y;
    } else {
      C[lmi(l + 1, l + 1)] = t * (x * C[lmi(l, l)] - y * C[lmi(l, -l)]);
      C[lmi(l + 1, -(l + 1))] = t * (y * C[lmi(l, l)] + x * C[lmi(l, -l)]);
    }
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      double v = c_harm.mid_b[l][m + SEA_LMAX] * z * C[lmi(l, m)];
      if (l >= 1 && m >= -(l - 1) && m <= l - 1)
        v -= c_harm.mid_c[l][m + SEA_LMAX] * r2 * C[lmi(l - 1, m)];
      C[lmi(l + 1, m)] = v;
    }
  }
}

// Multipole potential sum_lm Q_lm C_lm(r)/r^(2l+1) at r = (x, y, z) != 0,
// through the irregular harmonics I_lm = C_lm / r^(2l+1), which obey the
// same recurrence scaled by 1/r^2 per level (I_00 = 1/r).  Q in shared or
// global memory, zero beyond the requested l_max.
__device__ __forceinline__ double me_potential(const double* __restrict__ Q, double x,
                                               double y, double z) {
  const double r2 = x * x + y * y + z * z;
  const double ir2 = 1.0 / r2;
  double I[SEA_NQ];
  I[0] = sqrt(ir2);
  double v = Q[0] * I[0];
#pragma unroll
  for (int l = 0; l < SEA_LMAX; ++l) {
    const double t = c_harm.top[l] * ir2;
    if (l == 0) {
      I[lmi(1, 1)] = t * x * I[0];
      I[lmi(1, -1)] = t * y * I[0];
    } else {
      I[lmi(l + 1, l + 1)] = t * (x * I[lmi(l, l)] - y * I[lmi(l, -l)]);
      I[lmi(l + 1, -(l + 1))] = t * (y * I[lmi(l, l)] + x * I[lmi(l, -l)]);
    }
#pragma unroll
    for (int m = -l; m <= l; ++m) {
      double u = c_harm.mid_b[l][m + SEA_LMAX] * z * I[lmi(l, m)];
      if (l >= 1 && m >= -(l - 1) && m <= l - 1) u -= c_harm.mid_c[l][m + SEA_LMAX] * I[lmi(l - 1, m)];
      I[lmi(l + 1, m)] = u * ir2;
    }
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m) v = fma(Q[lmi(l + 1, m)], I[lmi(l + 1, m)], v);
  }
  return v;
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
  bool have_phi = false, have_vxx = false, have_ace = false;

  // plan sizes (host copies)
  int P = 0, Pproto = 0, E = 0;
  long long U = 0, WC = 0, max_window = 0;

  sea_stats stats{};

  // device buffers
  SeaBuf phi, vxx_dev, psi_dev, out_dev;
  SeaBuf rowsum, colsum, marg, box;
  SeaBuf cand_flag, cand_geom, list_a, list_b, cand_S, counts;
  SeaBuf pinfo, pS, psize, voff, order, Q, epair, iters;
  SeaBuf vbuf, bbuf, rbuf, pbuf, qbuf;
  SeaBuf eptr, eent, ewin, coff, cbuf;
  SeaBuf status, exx_dev, queue;
  // ACE
  SeaBuf tmask, tptr_o, tlist_o, tslot_o, tptr_t, tlist_t, partial, Mbuf, Abuf, Lbuf, Linv,
      Gbuf, Hbuf, Hbuf2;
  int n_tiles = 0, tile_inc = 0, max_tile_list = 0;

  long long launches = 0;
  cudaEvent_t ev[10] = {};
};

// Host-side helpers implemented in api.cu.
sea_status sea_fail(sea_ctx* c, sea_status s, const char* msg);
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

// Launch wrappers (each file implements its own).
namespace sea {
cudaError_t launch_plan_boxes(sea_ctx* c);
cudaError_t launch_plan_pairs(sea_ctx* c);
cudaError_t launch_pair_setup(sea_ctx* c);
cudaError_t launch_cg(sea_ctx* c);
cudaError_t launch_entries(sea_ctx* c);
cudaError_t launch_accumulate(sea_ctx* c, double* out);
cudaError_t launch_ace_build(sea_ctx* c);
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
