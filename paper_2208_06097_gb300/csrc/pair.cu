// pair.cu -- per-pair Poisson problems (Sec. II B: Eqs. pe, me, mepole).
//
// k_pair_setup (one CTA per pair): rho_ij = phi_i phi_j on Omega_ij, its
//   multipole moments about the box centre, the multipole potential at every
//   point outside the box that the 37-point stencil reaches (one coordinate
//   outside, by 1..6), and the right-hand side b = 4 pi rho + (stencil
//   weights x those boundary values).
// k_cg (persistent, longest pairs first): conjugate gradients for
//   -Lap_h v = b on the box with zero values outside, FP64, two block
//   reductions per iteration (warp shuffles, then warps in fixed order),
//   the 37-point O(h^12) operator written as 37 fused multiply-adds (on this
//   part the FP64 FMA pipe issues faster than FP64 add); then the pair
//   integral sum rho v dV of Eq. exxGen_mlwf.
#include "sea_internal.cuh"

namespace sea {

struct StencilW {
  double ax[3][SEA_FDP + 1];  // -c_k / h_a^2
  double center;              // -sum_a c_0 / h_a^2
  double rhs[3][SEA_FDP + 1]; // +c_k / h_a^2 (boundary values moved to b)
};

// Moments: acc[lm] += rho * C_lm(x, y, z), computed level by level.
__device__ __forceinline__ void moment_accumulate(double rho, double x, double y, double z,
                                                  double* acc) {
  const double r2 = x * x + y * y + z * z;
  double C[SEA_NQ];
  C[0] = 1.0;
  acc[0] += rho;
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
#pragma unroll
    for (int m = -(l + 1); m <= l + 1; ++m) acc[lmi(l + 1, m)] = fma(rho, C[lmi(l + 1, m)], acc[lmi(l + 1, m)]);
  }
}

__global__ void __launch_bounds__(256, 1)
    k_pair_setup(const double* __restrict__ phi, int nx, int ny, int nz,
                 const PairInfo* __restrict__ pinfo, const long long* __restrict__ voff,
                 double hx, double hy, double hz, double dV, int lmax, StencilW W,
                 double* __restrict__ bbuf, double* __restrict__ Qout) {
  const int p = blockIdx.x;
  const PairInfo P = pinfo[p];
  const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2];
  const int n = P.n;
  const size_t ng = (size_t)nx * ny * nz;
  const double* fi = phi + (size_t)P.i * ng;
  const double* fj = phi + (size_t)P.j * ng;
  double* b = bbuf + voff[p];
  const double cx = 0.5 * (ex - 1), cy = 0.5 * (ey - 1), cz = 0.5 * (ez - 1);

  __shared__ double red[8][SEA_NQ];
  __shared__ double Qs[SEA_NQ];

  double acc[SEA_NQ];
#pragma unroll
  for (int q = 0; q < SEA_NQ; ++q) acc[q] = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int x = t % ex, y = (t / ex) % ey, z = t / (ex * ey);
    const size_t g = ((size_t)wrapi(P.lo[2] + z, nz) * ny + wrapi(P.lo[1] + y, ny)) * nx +
                     wrapi(P.lo[0] + x, nx);
    const double rho = fi[g] * fj[g];
    b[t] = rho;
    moment_accumulate(rho, (x - cx) * hx, (y - cy) * hy, (z - cz) * hz, acc);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < SEA_NQ; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < SEA_NQ) {
    const int q = threadIdx.x;
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][q];
    int l = 0;
    while ((l + 1) * (l + 1) <= q) ++l;
    const double Q = (l <= lmax) ? s * dV : 0.0;
    Qs[q] = Q;
    Qout[(size_t)p * SEA_NQ + q] = Q;
  }
  const double fourpi = 4.0 * 3.14159265358979323846;
  for (int t = threadIdx.x; t < n; t += blockDim.x) b[t] *= fourpi;
  __syncthreads();

  // Boundary values along each axis, one thread per line of the box.
  const int e3[3] = {ex, ey, ez};
  const double h3[3] = {hx, hy, hz};
  const double c3[3] = {cx, cy, cz};
  for (int a = 0; a < 3; ++a) {
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    const int nl = e3[b1] * e3[b2];
    const int ea = e3[a];
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
      int u[3];
      u[b1] = line % e3[b1];
      u[b2] = line / e3[b1];
      double Glo[SEA_FDP + 1], Ghi[SEA_FDP + 1];
#pragma unroll
      for (int d = 1; d <= SEA_FDP; ++d) {
        double r[3];
        r[b1] = (u[b1] - c3[b1]) * h3[b1];
        r[b2] = (u[b2] - c3[b2]) * h3[b2];
        r[a] = (-d - c3[a]) * h3[a];
        Glo[d] = me_potential(Qs, r[0], r[1], r[2]);
        r[a] = (ea - 1 + d - c3[a]) * h3[a];
        Ghi[d] = me_potential(Qs, r[0], r[1], r[2]);
      }
      const int sa = a == 0 ? 1 : (a == 1 ? ex : ex * ey);
      int base = 0;
      {
        int uu[3] = {u[0], u[1], u[2]};
        uu[a] = 0;
        base = (uu[2] * ey + uu[1]) * ex + uu[0];
      }
      for (int ta = 0; ta < ea; ++ta) {
        if (ta >= SEA_FDP && ta < ea - SEA_FDP) continue;
        double add = 0.0;
#pragma unroll
        for (int k = 1; k <= SEA_FDP; ++k) {
          if (ta - k < 0) add += W.rhs[a][k] * Glo[k - ta];
          if (ta + k > ea - 1) add += W.rhs[a][k] * Ghi[ta + k - (ea - 1)];
        }
        b[base + ta * sa] += add;
      }
    }
    __syncthreads();
  }
}

// q = -Lap_h p at box point t = (x, y, z), zero outside the box.
__device__ __forceinline__ double neg_lap(const double* __restrict__ pv, int t, int x, int y,
                                          int z, int ex, int ey, int ez, const StencilW& W) {
  const int sy = ex, sz = ex * ey;
  double a0 = W.center * pv[t];
  double a1 = 0.0;
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const double L = (x - k >= 0) ? pv[t - k] : 0.0;
    const double R = (x + k < ex) ? pv[t + k] : 0.0;
    a0 = fma(W.ax[0][k], L, a0);
    a1 = fma(W.ax[0][k], R, a1);
  }
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const double L = (y - k >= 0) ? pv[t - k * sy] : 0.0;
    const double R = (y + k < ey) ? pv[t + k * sy] : 0.0;
    a0 = fma(W.ax[1][k], L, a0);
    a1 = fma(W.ax[1][k], R, a1);
  }
#pragma unroll
  for (int k = 1; k <= SEA_FDP; ++k) {
    const double L = (z - k >= 0) ? pv[t - k * sz] : 0.0;
    const double R = (z + k < ez) ? pv[t + k * sz] : 0.0;
    a0 = fma(W.ax[2][k], L, a0);
    a1 = fma(W.ax[2][k], R, a1);
  }
  return a0 + a1;
}

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
};

__global__ void __launch_bounds__(256) k_cg(CgArgs A, StencilW W) {
  __shared__ double red[2][32];
  __shared__ int s_item;
  const size_t ng = (size_t)A.nx * A.ny * A.nz;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= A.P) break;
    const int pidx = A.order[item];
    const PairInfo P = A.pinfo[pidx];
    const int ex = P.ext[0], ey = P.ext[1], ez = P.ext[2], n = P.n;
    const long long off = A.voff[pidx];
    double* x = A.x + off;
    const double* b = A.b + off;
    double* r = A.r + off;
    double* pv = A.p + off;
    double* q = A.q + off;

    double rr = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double bt = b[t];
      x[t] = 0.0;
      r[t] = bt;
      pv[t] = bt;
      rr = fma(bt, bt, rr);
    }
    rr = block_sum(rr, red[0]);
    const double bnorm = sqrt(rr);
    const double target =
        A.tol_mode == 0 ? A.tol * bnorm : A.tol * 4.0 * 3.14159265358979323846 * sqrt((double)n);
    int it = 0;
    bool done = sqrt(rr) <= target;
    while (!done && it < A.max_iter) {
      double pq = 0.0;
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int xx = t % ex, yy = (t / ex) % ey, zz = t / (ex * ey);
        const double qt = neg_lap(pv, t, xx, yy, zz, ex, ey, ez, W);
        q[t] = qt;
        pq = fma(pv[t], qt, pq);
      }
      pq = block_sum(pq, red[1]);
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
    // pair integral of Eq. exxGen_mlwf over Omega_ij
    const double* fi = A.phi + (size_t)P.i * ng;
    const double* fj = A.phi + (size_t)P.j * ng;
    double e = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int xx = t % ex, yy = (t / ex) % ey, zz = t / (ex * ey);
      const size_t g = ((size_t)wrapi(P.lo[2] + zz, A.nz) * A.ny + wrapi(P.lo[1] + yy, A.ny)) * A.nx +
                       wrapi(P.lo[0] + xx, A.nx);
      e = fma(fi[g] * fj[g], x[t], e);
    }
    e = block_sum(e, red[1]);
    if (threadIdx.x == 0) {
      A.epair[pidx] = e * A.dV;
      A.iters[pidx] = done ? it : -it;
      if (!done) atomicOr(A.status, SEA_FLAG_CG_CAP);
    }
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
  k_pair_setup<<<c->P, 256, 0, c->stream>>>(
      (const double*)c->phi.p, c->N[0], c->N[1], c->N[2], (const PairInfo*)c->pinfo.p,
      (const long long*)c->voff.p, c->h[0], c->h[1], c->h[2], c->dV, c->prm.lmax,
      make_weights(c), (double*)c->bbuf.p, (double*)c->Q.p);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_cg(sea_ctx* c) {
  if (c->P == 0) return cudaSuccess;
  int nsm = 0, occ = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg, 256, 0);
  if (occ < 1) occ = 1;
  const int grid = min(c->P, nsm * occ);
  cudaMemsetAsync(c->queue.p, 0, sizeof(int), c->stream);
  CgArgs A;
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
  k_cg<<<grid, 256, 0, c->stream>>>(A, make_weights(c));
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t upload_harmonics_pair() { return upload_harmonics_here(); }

}  // namespace sea
