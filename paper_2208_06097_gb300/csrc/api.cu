// api.cu -- the C ABI of libsea.so (declared in include/sea.h): context,
// parameters, workspace and the order of the device steps.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#include <new>

#include "sea_internal.cuh"

namespace sea {

// Coefficients of the rescaled solid-harmonic recurrences (see
// sea_internal.cuh).  From the Racah-normalized recurrences
//   C_{l+1,+-(l+1)} = t_l (x C_ll -+ y C_l,-l ...),  t_l = sqrt(2^[l=0] (2l+1)/(2l+2))
//   C_{l+1,m} = b_lm z C_lm - c_lm r^2 C_{l-1,m},
//   b_lm = (2l+1)/sqrt((l+m+1)(l-m+1)),  c_lm = sqrt((l+m)(l-m)/((l+m+1)(l-m+1))),
// the scaling kappa_lm = tau_|m| sigma_lm with tau_0 = 1, tau_{k+1} = t_k tau_k,
// sigma_{|m|,m} = 1, sigma_{l+1,m} = b_lm sigma_lm removes t and b; then
// gam_lm = c_lm sigma_{l-1,m} / sigma_{l+1,m}.
// The bit pattern of a double, for graph signatures.
uintptr_t bits_of(double v) {
  uintptr_t u = 0;
  memcpy(&u, &v, sizeof(double) < sizeof(u) ? sizeof(double) : sizeof(u));
  return u;
}

HarmCoef make_harmonic_coefficients() {
  HarmCoef h;
  memset(&h, 0, sizeof(h));
  double tau[SEA_LMAX + 1];
  tau[0] = 1.0;
  for (int k = 0; k < SEA_LMAX; ++k)
    tau[k + 1] = std::sqrt((k == 0 ? 2.0 : 1.0) * (2.0 * k + 1.0) / (2.0 * k + 2.0)) * tau[k];
  double sig[SEA_LMAX + 1][2 * SEA_LMAX + 1];
  for (int l = 0; l <= SEA_LMAX; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      if (l == am) {
        sig[l][m + SEA_LMAX] = 1.0;
      } else {
        const int lp = l - 1;  // sigma_{lp+1,m} = b_{lp,m} sigma_{lp,m}
        const double b = (2.0 * lp + 1.0) / std::sqrt((double)(lp + m + 1) * (double)(lp - m + 1));
        sig[l][m + SEA_LMAX] = b * sig[lp][m + SEA_LMAX];
      }
      const double kap = tau[am] * sig[l][m + SEA_LMAX];
      h.kap2[l * l + l + m] = kap * kap;
    }
  for (int l = 1; l < SEA_LMAX; ++l)
    for (int m = -(l - 1); m <= l - 1; ++m) {
      const double c = std::sqrt((double)(l + m) * (double)(l - m) /
                                 ((double)(l + m + 1) * (double)(l - m + 1)));
      h.gam[l][m + SEA_LMAX] = c * sig[l - 1][m + SEA_LMAX] / sig[l + 1][m + SEA_LMAX];
    }
  for (int l = 0; l < SEA_LMAX; ++l)
    for (int k = 0; k < 2 * SEA_LMAX + 1; ++k) {
      const float hi = (float)h.gam[l][k];
      h.gam_hi[l][k] = hi;
      h.gam_lo[l][k] = (float)(h.gam[l][k] - (double)hi);
    }
  // D_lm as polynomials: coefficient arrays P[a][b][c] of x^a y^b z^c, the
  // recurrence applied to them (multiplication by x, y, z, r^2 shifts them)
  constexpr int E = SEA_LMAX + 1;
  std::vector<double> P((size_t)SEA_NQ * E * E * E, 0.0);
  auto at = [&](int q, int a, int b, int c) -> double& {
    return P[(((size_t)q * E + a) * E + b) * E + c];
  };
  // dst += f * (x^dx y^dy z^dz) src
  auto add_shift = [&](int dst, int src, double f, int dx, int dy, int dz) {
    for (int a = 0; a + dx < E; ++a)
      for (int b = 0; b + dy < E; ++b)
        for (int c = 0; c + dz < E; ++c)
          if (at(src, a, b, c) != 0.0) at(dst, a + dx, b + dy, c + dz) += f * at(src, a, b, c);
  };
  at(0, 0, 0, 0) = 1.0;
  at(lmi(1, 1), 1, 0, 0) = 1.0;
  at(lmi(1, -1), 0, 1, 0) = 1.0;
  at(lmi(1, 0), 0, 0, 1) = 1.0;
  for (int l = 1; l < SEA_LMAX; ++l) {
    add_shift(lmi(l + 1, l + 1), lmi(l, l), 1.0, 1, 0, 0);
    add_shift(lmi(l + 1, l + 1), lmi(l, -l), -1.0, 0, 1, 0);
    add_shift(lmi(l + 1, -(l + 1)), lmi(l, l), 1.0, 0, 1, 0);
    add_shift(lmi(l + 1, -(l + 1)), lmi(l, -l), 1.0, 1, 0, 0);
    for (int m = -l; m <= l; ++m) {
      add_shift(lmi(l + 1, m), lmi(l, m), 1.0, 0, 0, 1);
      if (m >= -(l - 1) && m <= l - 1) {
        const double g = h.gam[l][m + SEA_LMAX];
        add_shift(lmi(l + 1, m), lmi(l - 1, m), -g, 2, 0, 0);
        add_shift(lmi(l + 1, m), lmi(l - 1, m), -g, 0, 2, 0);
        add_shift(lmi(l + 1, m), lmi(l - 1, m), -g, 0, 0, 2);
      }
    }
  }
  for (int l = 0; l <= SEA_LMAX; ++l)
    for (int m = -l; m <= l; ++m)
      for (int a = 0; a <= l; ++a)
        for (int b = 0; a + b <= l; ++b) h.cart[lmi(l, m)][a][b] = at(lmi(l, m), a, b, l - a - b);
  return h;
}

// Input check of sea_set_orbitals, one pass over the orbitals: every value
// finite, and part[o][b] = sum of phi_o^2 over chunk b of orbital o (grid
// blockIdx.x = chunk, blockIdx.y = orbital of the range).
#define SEA_NORM_CHUNKS 16
__global__ void __launch_bounds__(256)
    k_check_orbitals(const double* __restrict__ f, size_t ng, unsigned* __restrict__ st,
                     double* __restrict__ part) {
  __shared__ double red[32];
  const size_t chunk = (ng + SEA_NORM_CHUNKS - 1) / SEA_NORM_CHUNKS;
  const size_t b0 = chunk * blockIdx.x, b1 = min(ng, b0 + chunk);
  const double* fo = f + (size_t)blockIdx.y * ng;
  bool bad = false;
  double s = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const double v = fo[i];
    bad |= !isfinite(v);
    s = fma(v, v, s);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(st, SEA_FLAG_NONFINITE);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * SEA_NORM_CHUNKS + blockIdx.x] = s;
}

// |dV sum_b part[o][b] - 1| > tol for some orbital o: SEA_FLAG_NORM (the
// chunks added in index order).
__global__ void k_check_norms(const double* __restrict__ part, int n, double dV, double tol,
                              unsigned* __restrict__ st) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  double s = 0.0;
  for (int b = 0; b < SEA_NORM_CHUNKS; ++b) s += part[(size_t)o * SEA_NORM_CHUNKS + b];
  if (!(fabs(s * dV - 1.0) <= tol)) atomicOr(st, SEA_FLAG_NORM);
}

cudaError_t launch_plan_boxes(sea_ctx* c);
cudaError_t launch_plan_pairs(sea_ctx* c);
}  // namespace sea

// Second-derivative weights of the symmetric 13-point stencil by Fornberg's
// recursion (B. Fornberg, Math. Comp. 51, 699 (1988)) for nodes
// 0, 1, -1, ..., 6, -6; returns w[k], k = 0..6 (symmetric).
void sea::fornberg_weights(double* w) {
  const int np = 2 * SEA_FDP + 1, M = 2;
  double x[2 * SEA_FDP + 1];
  x[0] = 0.0;
  for (int k = 1; k <= SEA_FDP; ++k) {
    x[2 * k - 1] = k;
    x[2 * k] = -k;
  }
  double C[2 * SEA_FDP + 1][3];
  memset(C, 0, sizeof(C));
  C[0][0] = 1.0;
  double c1 = 1.0, c4 = x[0];
  for (int i = 1; i < np; ++i) {
    const int mn = i < M ? i : M;
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i];
    for (int j = 0; j < i; ++j) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k) C[i][k] = c1 * (k * C[i - 1][k - 1] - c5 * C[i - 1][k]) / c2;
        C[i][0] = -c1 * c5 * C[i - 1][0] / c2;
      }
      for (int k = mn; k >= 1; --k) C[j][k] = (c4 * C[j][k] - k * C[j][k - 1]) / c3;
      C[j][0] = c4 * C[j][0] / c3;
    }
    c1 = c2;
  }
  w[0] = C[0][2];
  for (int k = 1; k <= SEA_FDP; ++k) w[k] = 0.5 * (C[2 * k - 1][2] + C[2 * k][2]);
}

sea_status sea_fail(sea_ctx* c, sea_status s, const char* msg) {
  if (c) {
    snprintf(c->err, sizeof(c->err), "%s", msg);
    if (s == SEA_ERR_CUDA) c->poisoned = true;
  }
  return s;
}

bool sea_ensure(sea_ctx* c, SeaBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return true;
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return false;
  }
  b.bytes = want;
  return true;
}

static void release(SeaBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

#define SEA_CK(call, msg)                                                        \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      char b_[256];                                                              \
      snprintf(b_, sizeof(b_), "%s: %s", msg, cudaGetErrorString(e_));           \
      return sea_fail(c, SEA_ERR_CUDA, b_);                                      \
    }                                                                            \
  } while (0)

#define SEA_ALLOC(buf, bytes)                                                    \
  do {                                                                           \
    if (!sea_ensure(c, c->buf, (bytes))) return sea_fail(c, SEA_ERR_OOM, "device allocation failed: " #buf); \
  } while (0)

extern "C" {

void sea_default_params(sea_params* p) {
  if (!p) return;
  p->eps = std::pow(10.0, -3.5);
  p->delta = 1e-3;
  p->cg_tol = 1e-8;
  p->cg_tol_mode = 0;
  p->cg_max_iter = 5000;
  p->lmax = 6;
  p->fd_order = 12;
  p->self_scale = 2.0;
  p->precision = 0;
  p->warm_start = 0;
  p->timeout_ms = 0.0;
  p->ace_decomp = 0;
  p->orth_tol = 1e-6;
}

sea_status sea_create(const double cell[3], const int grid[3], const sea_params* p,
                      void* cuda_stream, sea_ctx** out) {
  if (!out || !cell || !grid) return SEA_ERR_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a) {
    if (!(cell[a] > 0.0) || !std::isfinite(cell[a])) return SEA_ERR_ARG;
    if (grid[a] < 8 || grid[a] > 1024) return SEA_ERR_ARG;
  }
  sea_params prm;
  sea_default_params(&prm);
  if (p) prm = *p;
  if (!(prm.eps >= 0.0 && prm.eps < 1.0) || !(prm.delta >= 0.0) || !(prm.cg_tol > 0.0) ||
      prm.cg_max_iter < 1 || prm.lmax < 0 || prm.lmax > SEA_LMAX || prm.fd_order != 12 ||
      prm.self_scale != 2.0 || (prm.precision != 0 && prm.precision != 1) || (prm.warm_start != 0 && prm.warm_start != 1) ||
      (prm.cg_tol_mode != 0 && prm.cg_tol_mode != 1) || prm.ace_decomp < 0 || prm.ace_decomp > 2 ||
      !(prm.timeout_ms >= 0.0 && prm.timeout_ms < 1e12) || !(prm.orth_tol >= 0.0))
    return SEA_ERR_ARG;
  sea_ctx* c = new (std::nothrow) sea_ctx();
  if (!c) return SEA_ERR_OOM;
  c->prm = prm;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return SEA_ERR_CUDA;
  }
  c->stream = (cudaStream_t)cuda_stream;
  for (int a = 0; a < 3; ++a) {
    c->cell[a] = cell[a];
    c->N[a] = grid[a];
    c->h[a] = cell[a] / grid[a];
  }
  c->dV = c->h[0] * c->h[1] * c->h[2];
  c->ng = (size_t)grid[0] * grid[1] * grid[2];
  double w[SEA_FDP + 1];
  sea::fornberg_weights(w);
  c->w_center = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double ih2 = 1.0 / (c->h[a] * c->h[a]);
    for (int k = 0; k <= SEA_FDP; ++k) c->w_ax[a][k] = -w[k] * ih2;
    c->w_center += -w[0] * ih2;
  }
  if (sea::upload_harmonics_pair() != cudaSuccess || sea::upload_harmonics_accum() != cudaSuccess) {
    delete c;
    return SEA_ERR_CUDA;
  }
  for (int k = 0; k < 16; ++k)
    if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
      sea_destroy(c);
      return SEA_ERR_CUDA;
    }
  for (int k = 0; k < 2; ++k)
    if (cudaStreamCreateWithFlags(&c->xfer[k], cudaStreamNonBlocking) != cudaSuccess) {
      sea_destroy(c);
      return SEA_ERR_CUDA;
    }
  for (int k = 0; k < 2 * SEA_XCHUNKS_MAX + 2; ++k)
    if (cudaEventCreateWithFlags(&c->xev[k], cudaEventDisableTiming) != cudaSuccess) {
      sea_destroy(c);
      return SEA_ERR_CUDA;
    }
  if (!sea_ensure(c, c->status, 64) || !sea_ensure(c, c->counts, 128) ||
      !sea_ensure(c, c->exx_dev, 64) || !sea_ensure(c, c->queue, 64)) {
    sea_destroy(c);
    return SEA_ERR_OOM;
  }
  *out = c;
  return SEA_OK;
}

sea_status sea_set_orbitals(sea_ctx* c, const double* phi, int n_orb, int on_device) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned by an earlier CUDA error");
  if (!phi || n_orb < 1 || n_orb > 4096) return sea_fail(c, SEA_ERR_ARG, "bad orbitals");
  c->have_phi = c->have_vxx = c->have_ace = false;
  const size_t bytes = (size_t)n_orb * c->ng * sizeof(double);
  SEA_ALLOC(phi, bytes);
  SEA_ALLOC(vxx_dev, bytes);
  c->n_orb = n_orb;
  const long long ncand = (long long)n_orb * (n_orb + 1) / 2;
  const int Nmax = std::max(c->N[0], std::max(c->N[1], c->N[2]));
  SEA_ALLOC(rowsum, (size_t)n_orb * c->N[2] * c->N[1] * sizeof(ulonglong2));
  SEA_ALLOC(colsum, (size_t)n_orb * c->N[2] * c->N[0] * sizeof(ulonglong2));
  SEA_ALLOC(marg, (size_t)n_orb * 3 * Nmax * sizeof(double));
  SEA_ALLOC(box, (size_t)n_orb * 6 * sizeof(int));
  SEA_ALLOC(cand_flag, ncand * sizeof(int));
  SEA_ALLOC(cand_geom, ncand * 9 * sizeof(int));
  SEA_ALLOC(list_a, ncand * sizeof(int));
  SEA_ALLOC(list_b, ncand * sizeof(int));
  SEA_ALLOC(cand_S, ncand * sizeof(double));
  SEA_ALLOC(pinfo, ncand * sizeof(PairInfo));
  SEA_ALLOC(pS, ncand * sizeof(double));
  SEA_ALLOC(psize, ncand * sizeof(int));
  SEA_ALLOC(voff, ncand * sizeof(long long));
  SEA_ALLOC(order, ncand * sizeof(int));
  SEA_ALLOC(eent, (size_t)(n_orb + 1) * sizeof(int));
  SEA_ALLOC(eptr, (size_t)(n_orb + 1) * sizeof(int));
  SEA_ALLOC(ewin, (size_t)2 * ncand * sizeof(Entry));
  SEA_ALLOC(coff, (size_t)2 * ncand * sizeof(long long));
  SEA_ALLOC(onorm, (size_t)n_orb * SEA_NORM_CHUNKS * sizeof(double));
  double* npart = (double*)c->onorm.p;
  SEA_CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), c->stream), "memset");
  double* pd = (double*)c->phi.p;
  if (on_device) {
    SEA_CK(cudaMemcpyAsync(pd, phi, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy orbitals");
    sea::k_check_orbitals<<<dim3(SEA_NORM_CHUNKS, n_orb), 256, 0, c->stream>>>(
        pd, c->ng, (unsigned*)c->status.p, npart);
    c->launches += 1;
  } else {
    // orbital ranges copied in on the copy stream, each checked on the
    // context stream once it has arrived
    const int nch = std::min(8, n_orb);
    cudaEvent_t ev_start = c->xev[2 * SEA_XCHUNKS_MAX];
    SEA_CK(cudaEventRecord(ev_start, c->stream), "event");
    SEA_CK(cudaStreamWaitEvent(c->xfer[0], ev_start, 0), "wait");
    for (int k = 0; k < nch; ++k) {
      const size_t o0 = (size_t)n_orb * k / nch, o1 = (size_t)n_orb * (k + 1) / nch;
      SEA_CK(cudaMemcpyAsync(pd + o0 * c->ng, phi + o0 * c->ng, (o1 - o0) * c->ng * sizeof(double),
                             cudaMemcpyHostToDevice, c->xfer[0]),
             "copy orbitals");
      SEA_CK(cudaEventRecord(c->xev[k], c->xfer[0]), "event");
    }
    for (int k = 0; k < nch; ++k) {
      const size_t o0 = (size_t)n_orb * k / nch, o1 = (size_t)n_orb * (k + 1) / nch;
      SEA_CK(cudaStreamWaitEvent(c->stream, c->xev[k], 0), "wait");
      sea::k_check_orbitals<<<dim3(SEA_NORM_CHUNKS, (unsigned)(o1 - o0)), 256, 0, c->stream>>>(
          pd + o0 * c->ng, c->ng, (unsigned*)c->status.p, npart + o0 * SEA_NORM_CHUNKS);
      c->launches += 1;
    }
  }
  if (c->prm.orth_tol > 0.0) {
    sea::k_check_norms<<<(n_orb + 127) / 128, 128, 0, c->stream>>>(npart, n_orb, c->dV,
                                                                    c->prm.orth_tol,
                                                                    (unsigned*)c->status.p);
    c->launches += 1;
  }
  SEA_CK(cudaGetLastError(), "input check");
  unsigned st = 0;
  SEA_CK(cudaMemcpyAsync(&st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
         "status");
  SEA_CK(cudaStreamSynchronize(c->stream), "set_orbitals");
  if (st & SEA_FLAG_NONFINITE) return sea_fail(c, SEA_ERR_INPUT, "orbitals hold non-finite values");
  if (st & SEA_FLAG_NORM)
    return sea_fail(c, SEA_ERR_INPUT, "an orbital's norm <phi|phi> differs from 1 by more than orth_tol");
  c->have_phi = true;
  c->stats.n_orb = n_orb;
  return SEA_OK;
}

sea_status sea_scdm(sea_ctx* c, const double* phi, int n_orb, int on_device, double* U, int* cols) {
  if (!c) return SEA_ERR_ARG;
  const sea_status st0 = sea_set_orbitals(c, phi, n_orb, on_device);
  if (st0 != SEA_OK) return st0;
  c->have_phi = false;
  const size_t nn = (size_t)n_orb * n_orb;
  SEA_ALLOC(scdm_u, nn * sizeof(double));
  SEA_ALLOC(scdm_c, (size_t)n_orb * sizeof(long long));
  SEA_CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), c->stream), "memset");
  const cudaError_t e = sea::launch_scdm(c, (double*)c->scdm_u.p, (long long*)c->scdm_c.p);
  if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "SCDM workspace");
  SEA_CK(e, "scdm");
  std::vector<long long> hc(n_orb);
  unsigned st = 0;
  if (U) SEA_CK(cudaMemcpyAsync(U, c->scdm_u.p, nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy U");
  SEA_CK(cudaMemcpyAsync(hc.data(), c->scdm_c.p, (size_t)n_orb * sizeof(long long), cudaMemcpyDeviceToHost,
                         c->stream),
         "copy pivots");
  SEA_CK(cudaMemcpyAsync(&st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "status");
  SEA_CK(cudaStreamSynchronize(c->stream), "scdm");
  if (st & SEA_FLAG_NOT_PD) return sea_fail(c, SEA_ERR_INPUT, "orbitals are rank deficient (SCDM pivot of zero norm)");
  if (cols)
    for (int k = 0; k < n_orb; ++k) cols[k] = (int)hc[k];
  c->have_phi = true;
  return SEA_OK;
}

sea_status sea_apply_vxx(sea_ctx* c, double* vxx_phi, int on_device, double* exx) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned by an earlier CUDA error");
  if (!c->have_phi) return sea_fail(c, SEA_ERR_STATE, "sea_set_orbitals first");
  if (!vxx_phi) return sea_fail(c, SEA_ERR_ARG, "vxx_phi is NULL");
  c->have_vxx = c->have_ace = false;
  sea::Trace tr("sea_apply_vxx");
  tr.stage("plan");
  SEA_CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), c->stream), "memset");
  SEA_CK(cudaEventRecord(c->ev[0], c->stream), "event");
  {
    // the plan: a fixed launch sequence for the context's sizes and buffers
    const std::vector<uintptr_t> sig = {
        (uintptr_t)c->n_orb, (uintptr_t)c->N[0], (uintptr_t)c->N[1], (uintptr_t)c->N[2],
        (uintptr_t)c->device, sea::bits_of(c->prm.eps), sea::bits_of(c->prm.delta),
        sea::bits_of(c->dV),
        (uintptr_t)c->phi.p, (uintptr_t)c->rowsum.p, (uintptr_t)c->colsum.p, (uintptr_t)c->marg.p,
        (uintptr_t)c->box.p, (uintptr_t)c->cand_flag.p, (uintptr_t)c->cand_geom.p,
        (uintptr_t)c->list_a.p, (uintptr_t)c->list_b.p, (uintptr_t)c->cand_S.p,
        (uintptr_t)c->counts.p, (uintptr_t)c->pinfo.p, (uintptr_t)c->pS.p, (uintptr_t)c->psize.p,
        (uintptr_t)c->voff.p, (uintptr_t)c->order.p, (uintptr_t)c->eent.p, (uintptr_t)c->eptr.p,
        (uintptr_t)c->ewin.p, (uintptr_t)c->coff.p};
    SEA_CK(run_graph(c, c->g_plan, sig,
                          [&]() {
                            cudaError_t e = sea::launch_plan_boxes(c);
                            if (e == cudaSuccess) e = sea::launch_plan_pairs(c);
                            if (e == cudaSuccess) e = sea::launch_entries(c);
                            return e;
                          }),
           "plan");
  }
  int hc[16];
  SEA_CK(cudaMemcpyAsync(hc, c->counts.p, sizeof(hc), cudaMemcpyDeviceToHost, c->stream), "counts");
  if (!on_device) {  // entry offsets: the output is produced and copied out by orbital ranges
    c->h_eptr.resize((size_t)c->n_orb + 1);
    SEA_CK(cudaMemcpyAsync(c->h_eptr.data(), c->eptr.p, ((size_t)c->n_orb + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, c->stream),
           "entry offsets");
  }
  SEA_CK(cudaStreamSynchronize(c->stream), "plan");
  c->Pproto = hc[0];
  c->P = hc[1];
  c->E = hc[2];
  memcpy(&c->U, hc + 4, sizeof(long long));
  memcpy(&c->WC, hc + 6, sizeof(long long));
  memcpy(&c->max_window, hc + 8, sizeof(long long));
  c->cg_pad_max = hc[10];
  SEA_CK(cudaEventRecord(c->ev[1], c->stream), "event");
  const size_t U = (size_t)std::max<long long>(c->U, 1);
  SEA_ALLOC(vbuf, U * sizeof(double));
  SEA_ALLOC(bbuf, U * sizeof(double));
  SEA_ALLOC(rbuf, U * sizeof(double));
  SEA_ALLOC(pbuf, U * sizeof(double));
  SEA_ALLOC(qbuf, U * sizeof(double));
  SEA_ALLOC(cbuf, (size_t)std::max<long long>(c->WC, 1) * sizeof(double));
  SEA_ALLOC(Q, (size_t)std::max(c->P, 1) * SEA_QSTRIDE * sizeof(double));
  SEA_ALLOC(epair, (size_t)std::max(c->P, 1) * sizeof(double));
  SEA_ALLOC(iters, (size_t)std::max(c->P, 1) * sizeof(int));
  c->lists_ready = false;
  tr.stage("pair setup");
  SEA_CK(sea::launch_pair_setup(c), "pair setup");
  c->cg_warm = false;
  if (c->prm.warm_start == 1) {  // learned initial guesses (the model's time counts as setup)
    if (!c->unet) return sea_fail(c, SEA_ERR_STATE, "warm_start = 1 needs sea_unet_attach");
    tr.stage("warm start");
    const cudaError_t e = sea::launch_warm_start(c);
    if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "warm-start workspace");
    SEA_CK(e, "warm start");
    c->cg_warm = true;
  }
  SEA_CK(cudaEventRecord(c->ev[2], c->stream), "event");
  tr.stage("cg");
  SEA_CK(sea::launch_cg(c), "cg");
  // W's tile lists for the ACE build follow from the plan alone: formed on
  // the second side stream, on the SMs that the CG's last pairs leave idle
  // (their counts come back with this call's results)
  {
    const cudaError_t e = sea::launch_ace_lists(c, c->xfer[1]);
    if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "ACE tile lists");
    SEA_CK(e, "ACE tile lists");
  }
  SEA_CK(sea::launch_contrib_far(c, c->ev[2]), "far field");
  SEA_CK(cudaEventRecord(c->ev[3], c->stream), "event");
  // E_xx and the CG statistics need the pair energies only: beside the far
  // field and the accumulation, after the lists on the same side stream
  SEA_CK(cudaStreamWaitEvent(c->xfer[1], c->ev[3], 0), "wait");
  SEA_CK(sea::launch_exx(c, c->xfer[1]), "exx");
  SEA_CK(cudaEventRecord(c->xev[2], c->xfer[1]), "event");
  tr.stage("far field and accumulation");
  double* vd = (double*)c->vxx_dev.p;
  if (on_device) {
    SEA_CK(sea::launch_accumulate(c, vd, vxx_phi, false), "accumulate");
    SEA_CK(cudaEventRecord(c->ev[4], c->stream), "event");
  } else {
    // Host output: orbital ranges are finished and copied out one after
    // another, the copy of one range overlapping the kernels of the next.
    const int nch = std::min(8, c->n_orb);
    cudaEvent_t ev_start = c->xev[2 * SEA_XCHUNKS_MAX];
    cudaEvent_t ev_out = c->xev[2 * SEA_XCHUNKS_MAX + 1];
    SEA_CK(cudaEventRecord(ev_start, c->stream), "event");
    SEA_CK(cudaStreamWaitEvent(c->xfer[1], ev_start, 0), "wait");
    for (int k = 0; k < nch; ++k) {
      const int o0 = (int)((long long)c->n_orb * k / nch);
      const int o1 = (int)((long long)c->n_orb * (k + 1) / nch);
      SEA_CK(sea::launch_accumulate_range(c, vd, o0, o1, c->h_eptr[o0], c->h_eptr[o1]),
             "accumulate");
      SEA_CK(cudaEventRecord(c->xev[SEA_XCHUNKS_MAX + k], c->stream), "event");
      SEA_CK(cudaStreamWaitEvent(c->xfer[1], c->xev[SEA_XCHUNKS_MAX + k], 0), "wait");
      SEA_CK(cudaMemcpyAsync(vxx_phi + (size_t)o0 * c->ng, vd + (size_t)o0 * c->ng,
                             (size_t)(o1 - o0) * c->ng * sizeof(double), cudaMemcpyDeviceToHost,
                             c->xfer[1]),
             "copy V_xx phi");
    }
    SEA_CK(cudaEventRecord(c->ev[4], c->stream), "event");
    SEA_CK(cudaEventRecord(ev_out, c->xfer[1]), "event");
    SEA_CK(cudaStreamWaitEvent(c->stream, ev_out, 0), "wait");
  }
  struct {
    double res[5];
    unsigned st;
    int lists[3];
  } r;
  SEA_CK(cudaStreamWaitEvent(c->stream, c->xev[2], 0), "wait");
  SEA_CK(cudaMemcpyAsync(r.res, c->exx_dev.p, sizeof(r.res), cudaMemcpyDeviceToHost, c->stream),
         "exx");
  SEA_CK(cudaMemcpyAsync(&r.st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
         "status");
  SEA_CK(cudaMemcpyAsync(r.lists, (int*)c->counts.p + 10, sizeof(r.lists), cudaMemcpyDeviceToHost,
                         c->stream),
         "list counts");
  SEA_CK(cudaStreamSynchronize(c->stream), "apply_vxx");
  c->tile_inc = r.lists[0];
  c->max_tile_list = r.lists[2];
  c->lists_ready = true;
  float t01 = 0, t12 = 0, t23 = 0, t34 = 0;
  cudaEventElapsedTime(&t01, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&t12, c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&t23, c->ev[2], c->ev[3]);
  cudaEventElapsedTime(&t34, c->ev[3], c->ev[4]);
  c->stats.ms_plan = t01;
  c->stats.ms_setup = t12;
  c->stats.ms_cg = t23;
  c->stats.ms_accumulate = t34;
  c->stats.n_pairs = c->P;
  c->stats.n_proto_pairs = c->Pproto;
  c->stats.n_unknowns = c->U;
  c->stats.n_window_points = c->WC;
  c->stats.exx = r.res[0];
  c->stats.cg_unknown_iters = (long long)r.res[1];
  c->stats.cg_iters_min = (int)r.res[2];
  c->stats.cg_iters_max = (int)r.res[3];
  c->stats.cg_iters_mean = r.res[4];
  if (exx) *exx = r.res[0];
  if (r.st & SEA_FLAG_WAIT)
    return sea_fail(c, SEA_ERR_CUDA, "a tensor-core completion wait timed out (warm start)");
  if (r.st & SEA_FLAG_TIMEOUT)
    return sea_fail(c, SEA_ERR_TIMEOUT,
                    "the CG time budget (timeout_ms) was spent before every pair was solved");
  c->have_vxx = true;
  if (r.st & SEA_FLAG_CG_CAP)
    return sea_fail(c, SEA_ERR_CG_NOT_CONVERGED, "a pair's CG reached cg_max_iter");
  return SEA_OK;
}

static sea_status build_ace_common(sea_ctx* c) {
  c->have_ace = false;
  c->ace_eigen = false;
  c->stats.ace_eigen = 0;
  c->stats.ace_eigen_sweeps = 0;
  c->stats.ace_negative_eigenvalues = 0;
  c->stats.ace_dropped_eigenvalues = 0;
  sea::Trace tr("sea_build_ace");
  tr.stage("M and Cholesky");
  SEA_CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), c->stream), "memset");
  SEA_CK(cudaEventRecord(c->ev[5], c->stream), "event");
  cudaError_t e = sea::launch_ace_build(c);
  if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "ACE workspace");
  SEA_CK(e, "ace build");
  // the status and, for the Cholesky form, E_xx^ACE in one read-back
  struct {
    double exx_ace;
    unsigned st;
  } rb = {0.0, 0u};
  SEA_CK(cudaEventRecord(c->ev[6], c->stream), "event");
  SEA_CK(cudaMemcpyAsync(&rb.exx_ace, (double*)c->exx_dev.p + SEA_EXX_ACE_SLOT, sizeof(double),
                         cudaMemcpyDeviceToHost, c->stream),
         "exx_ace");
  SEA_CK(cudaMemcpyAsync(&rb.st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
         "status");
  SEA_CK(cudaStreamSynchronize(c->stream), "build_ace");
  if (rb.st & SEA_FLAG_WAIT)
    return sea_fail(c, SEA_ERR_CUDA, "a bounded completion wait timed out (ACE build)");
  const bool not_pd = (rb.st & SEA_FLAG_NOT_PD) != 0;
  if ((not_pd && c->prm.ace_decomp == 0) || c->prm.ace_decomp == 2) {
    tr.stage("eigen-decomposition");
    e = sea::launch_ace_eigen(c);
    if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "ACE eigen workspace");
    SEA_CK(e, "ace eigen form");
    c->stats.ace_eigen = 1;
    SEA_CK(cudaEventRecord(c->ev[6], c->stream), "event");
    SEA_CK(cudaMemcpyAsync(&rb.exx_ace, (double*)c->exx_dev.p + SEA_EXX_ACE_SLOT, sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream),
           "exx_ace");
    SEA_CK(cudaStreamSynchronize(c->stream), "build_ace");
  } else if (not_pd) {
    return sea_fail(c, SEA_ERR_NOT_PD, "-Mbar is not positive definite");
  }
  c->stats.exx_ace = rb.exx_ace;
  float t = 0;
  cudaEventElapsedTime(&t, c->ev[5], c->ev[6]);
  c->stats.ms_ace_build = t;
  cudaEventElapsedTime(&t, c->ev[10], c->ev[11]);
  c->stats.ms_gram_build = t;
  c->stats.ace_support_points = (long long)c->tile_inc * 128;
  c->stats.ace_max_tile_list = c->max_tile_list;
  if (c->ace_eigen && c->stats.ace_dropped_eigenvalues == c->n_orb)
    return sea_fail(c, SEA_ERR_NOT_PD, "-Mbar is zero");
  c->have_ace = true;
  return SEA_OK;
}

sea_status sea_build_ace(sea_ctx* c) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned by an earlier CUDA error");
  if (!c->have_vxx) return sea_fail(c, SEA_ERR_STATE, "sea_apply_vxx first");
  c->w_dense = false;
  return build_ace_common(c);
}

sea_status sea_build_ace_from(sea_ctx* c, const double* W, int on_device) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned by an earlier CUDA error");
  if (!c->have_phi) return sea_fail(c, SEA_ERR_STATE, "sea_set_orbitals first");
  if (!W) return sea_fail(c, SEA_ERR_ARG, "W is NULL");
  const size_t bytes = (size_t)c->n_orb * c->ng * sizeof(double);
  SEA_CK(cudaMemcpyAsync(c->vxx_dev.p, W, bytes,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
         "copy W");
  c->have_vxx = false;  // the context's W is no longer an apply_vxx result
  c->w_dense = true;
  return build_ace_common(c);
}

sea_status sea_apply_ace(sea_ctx* c, const double* psi, int n_vec, double* out, int on_device) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned by an earlier CUDA error");
  if (!c->have_ace) return sea_fail(c, SEA_ERR_STATE, "sea_build_ace first");
  if (!psi || !out || n_vec < 1) return sea_fail(c, SEA_ERR_ARG, "bad psi/out");
  sea::Trace tr("sea_apply_ace");
  const size_t bytes = (size_t)n_vec * c->ng * sizeof(double);
  if (on_device) {
    SEA_CK(cudaEventRecord(c->ev[7], c->stream), "event");
    cudaError_t e = sea::launch_ace_apply(c, psi, n_vec, out);
    if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "ACE apply workspace");
    SEA_CK(e, "ace apply");
    SEA_CK(cudaEventRecord(c->ev[8], c->stream), "event");
    c->apply_timed = true;
    return SEA_OK;
  }
  // Host buffers: the vectors are independent, so the call runs in chunks
  // of vectors: chunk k is copied in on one copy stream, applied on the
  // context stream and copied out on the other copy stream, so the two
  // transfer directions and the kernels overlap.
  SEA_ALLOC(psi_dev, bytes);
  SEA_ALLOC(out_dev, bytes);
  // chunk starts: a half-size first and last chunk (the copy-in before the
  // first kernels and the copy-out after the last ones are not overlapped)
  const int per = std::max(32, (n_vec + SEA_XCHUNKS_MAX - 1) / SEA_XCHUNKS_MAX);
  std::vector<int> cs;
  {
    const int h = per / 2;
    int v = 0;
    cs.push_back(0);
    if (n_vec > 2 * per && (n_vec - 2 * h) / per + 3 <= SEA_XCHUNKS_MAX) {
      v = h;
      cs.push_back(v);
      while (n_vec - h - v >= per) {
        v += per;
        cs.push_back(v);
      }
      if (n_vec - h > v) cs.push_back(n_vec - h);
    } else {
      while (v + per < n_vec) {
        v += per;
        cs.push_back(v);
      }
    }
    cs.push_back(n_vec);
  }
  const int nch = (int)cs.size() - 1;
  double* pd = (double*)c->psi_dev.p;
  double* od = (double*)c->out_dev.p;
  cudaEvent_t* evH = c->xev;             // chunk k copied in
  cudaEvent_t* evC = c->xev + SEA_XCHUNKS_MAX;  // chunk k applied
  cudaEvent_t ev_start = c->xev[2 * SEA_XCHUNKS_MAX];
  cudaEvent_t ev_out = c->xev[2 * SEA_XCHUNKS_MAX + 1];
  SEA_CK(cudaEventRecord(ev_start, c->stream), "event");
  SEA_CK(cudaStreamWaitEvent(c->xfer[0], ev_start, 0), "wait");
  SEA_CK(cudaStreamWaitEvent(c->xfer[1], ev_start, 0), "wait");
  for (int k = 0; k < nch; ++k) {
    const size_t v0 = (size_t)cs[k], nv = (size_t)(cs[k + 1] - cs[k]);
    SEA_CK(cudaMemcpyAsync(pd + v0 * c->ng, psi + v0 * c->ng, nv * c->ng * sizeof(double),
                           cudaMemcpyHostToDevice, c->xfer[0]),
           "copy psi");
    SEA_CK(cudaEventRecord(evH[k], c->xfer[0]), "event");
  }
  SEA_CK(cudaEventRecord(c->ev[7], c->stream), "event");
  for (int k = 0; k < nch; ++k) {
    const size_t v0 = (size_t)cs[k], nv = (size_t)(cs[k + 1] - cs[k]);
    SEA_CK(cudaStreamWaitEvent(c->stream, evH[k], 0), "wait");
    cudaError_t e = sea::launch_ace_apply(c, pd + v0 * c->ng, (int)nv, od + v0 * c->ng);
    if (e == cudaErrorMemoryAllocation) return sea_fail(c, SEA_ERR_OOM, "ACE apply workspace");
    SEA_CK(e, "ace apply");
    SEA_CK(cudaEventRecord(evC[k], c->stream), "event");
    SEA_CK(cudaStreamWaitEvent(c->xfer[1], evC[k], 0), "wait");
    SEA_CK(cudaMemcpyAsync(out + v0 * c->ng, od + v0 * c->ng, nv * c->ng * sizeof(double),
                           cudaMemcpyDeviceToHost, c->xfer[1]),
           "copy out");
  }
  SEA_CK(cudaEventRecord(c->ev[8], c->stream), "event");
  SEA_CK(cudaEventRecord(ev_out, c->xfer[1]), "event");
  SEA_CK(cudaStreamWaitEvent(c->stream, ev_out, 0), "wait");
  unsigned st = 0;
  SEA_CK(cudaMemcpyAsync(&st, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
         "status");
  SEA_CK(cudaStreamSynchronize(c->stream), "apply_ace");
  c->apply_timed = true;
  if (st & SEA_FLAG_WAIT)
    return sea_fail(c, SEA_ERR_CUDA, "a tensor-core completion wait timed out (ACE apply)");
  return SEA_OK;
}

sea_status sea_get_ace_matrices(sea_ctx* c, double* M, double* L, int on_device) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned");
  if (!c->have_ace) return sea_fail(c, SEA_ERR_STATE, "sea_build_ace first");
  const size_t bytes = (size_t)c->n_orb * c->n_orb * sizeof(double);
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (M) SEA_CK(cudaMemcpyAsync(M, c->Mbuf.p, bytes, k, c->stream), "copy M");
  if (L) SEA_CK(cudaMemcpyAsync(L, c->Lbuf.p, bytes, k, c->stream), "copy L");
  SEA_CK(cudaStreamSynchronize(c->stream), "get_ace_matrices");
  return SEA_OK;
}

sea_status sea_get_ace_vectors(sea_ctx* c, double* xi, int on_device) {
  if (!c) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned");
  if (!c->have_ace) return sea_fail(c, SEA_ERR_STATE, "sea_build_ace first");
  if (c->ace_eigen) return sea_fail(c, SEA_ERR_STATE, "the eigen form's ACE vectors may be complex");
  if (!xi) return sea_fail(c, SEA_ERR_ARG, "xi is NULL");
  const size_t bytes = (size_t)c->n_orb * c->ng * sizeof(double);
  double* dst = xi;
  if (!on_device) {
    SEA_ALLOC(out_dev, bytes);
    dst = (double*)c->out_dev.p;
  }
  SEA_CK(sea::launch_ace_vectors(c, dst), "ace vectors");
  if (!on_device) SEA_CK(cudaMemcpyAsync(xi, dst, bytes, cudaMemcpyDeviceToHost, c->stream), "copy xi");
  SEA_CK(cudaStreamSynchronize(c->stream), "get_ace_vectors");
  return SEA_OK;
}

sea_status sea_get_plan(sea_ctx* c, int* box, int* n_pairs, int max_pairs, int* pairs, int* lo,
                        int* ext, double* S, int* iters, double* epair) {
  if (!c || !n_pairs) return SEA_ERR_ARG;
  if (c->poisoned) return sea_fail(c, SEA_ERR_STATE, "context poisoned");
  if (!c->have_vxx) return sea_fail(c, SEA_ERR_STATE, "sea_apply_vxx first");
  *n_pairs = c->P;
  if (box)
    SEA_CK(cudaMemcpyAsync(box, c->box.p, (size_t)c->n_orb * 6 * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream),
           "copy box");
  const int m = std::min(max_pairs, c->P);
  if (m > 0) {
    PairInfo* pi = (PairInfo*)malloc((size_t)m * sizeof(PairInfo));
    if (!pi) return sea_fail(c, SEA_ERR_OOM, "host allocation");
    cudaError_t e = cudaMemcpyAsync(pi, c->pinfo.p, (size_t)m * sizeof(PairInfo),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && S)
      e = cudaMemcpyAsync(S, c->pS.p, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && iters)
      e = cudaMemcpyAsync(iters, c->iters.p, (size_t)m * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && epair)
      e = cudaMemcpyAsync(epair, c->epair.p, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      free(pi);
      SEA_CK(e, "copy plan");
    }
    for (int p = 0; p < m; ++p) {
      if (pairs) {
        pairs[2 * p] = pi[p].i;
        pairs[2 * p + 1] = pi[p].j;
      }
      for (int a = 0; a < 3; ++a) {
        if (lo) lo[3 * p + a] = pi[p].lo[a];
        if (ext) ext[3 * p + a] = pi[p].ext[a];
      }
    }
    free(pi);
  }
  SEA_CK(cudaStreamSynchronize(c->stream), "get_plan");
  return SEA_OK;
}

sea_status sea_poisson_batch(const double h[3], int n_box, const int* ext, const double* rhs,
                             double* x, double tol, int tol_mode, int max_iter, int* iters,
                             void* cuda_stream) {
  if (!h || n_box < 0 || (n_box > 0 && (!ext || !rhs || !x))) return SEA_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!(h[a] > 0.0)) return SEA_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 1 || (tol_mode != 0 && tol_mode != 1)) return SEA_ERR_ARG;
  if (n_box == 0) return SEA_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return SEA_ERR_CUDA;
  PairInfo* hb = (PairInfo*)malloc((size_t)n_box * sizeof(PairInfo));
  long long* ho = (long long*)malloc((size_t)n_box * sizeof(long long));
  int* hord = (int*)malloc((size_t)n_box * sizeof(int));
  if (!hb || !ho || !hord) {
    free(hb);
    free(ho);
    free(hord);
    return SEA_ERR_OOM;
  }
  long long tot = 0;
  sea_status rs = SEA_OK;
  for (int b = 0; b < n_box && rs == SEA_OK; ++b) {
    PairInfo P;
    memset(&P, 0, sizeof(P));
    for (int a = 0; a < 3; ++a) {
      P.ext[a] = ext[3 * b + a];
      if (P.ext[a] < 1 || P.ext[a] > 1024) rs = SEA_ERR_ARG;
    }
    P.n = P.ext[0] * P.ext[1] * P.ext[2];
    hb[b] = P;
    ho[b] = tot;
    tot += P.n;
    hord[b] = b;
  }
  if (rs != SEA_OK) {
    free(hb);
    free(ho);
    free(hord);
    return rs;
  }
  // longest boxes first (ties by index).  k_noalloc_order (noalloc.cu) ranks
  // the boxes of sea_poisson_batch_noalloc the same way; the two orders must
  // stay identical, since the solutions and iteration counts of the two entry
  // points are compared bit for bit.
  std::stable_sort(hord, hord + n_box, [&](int a, int b) { return hb[a].n > hb[b].n; });
  void* dev = nullptr;
  const size_t bytes = (size_t)n_box * (sizeof(PairInfo) + sizeof(long long) + 2 * sizeof(int)) +
                       3 * (size_t)tot * sizeof(double) + 64;
  if (cudaMalloc(&dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    free(hb);
    free(ho);
    free(hord);
    return SEA_ERR_OOM;
  }
  char* q = (char*)dev;
  double* r = (double*)q;
  double* pp = r + tot;
  double* qq = pp + tot;
  q = (char*)(qq + tot);
  long long* dvoff = (long long*)q;
  PairInfo* dbox = (PairInfo*)(dvoff + n_box);
  int* dord = (int*)(dbox + n_box);
  int* dit = dord + n_box;
  unsigned* dst = (unsigned*)(dit + n_box);
  int* dq = (int*)(dst + 1);
  cudaError_t e = cudaMemcpyAsync(dvoff, ho, n_box * sizeof(long long), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbox, hb, n_box * sizeof(PairInfo), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dord, hord, n_box * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, sizeof(unsigned), st);
  if (e == cudaSuccess)
    e = sea::launch_cg_boxes(st, device, h, n_box, dbox, dvoff, dord, rhs, x, r, pp, qq, dit, dst,
                             dq, tol, tol_mode, max_iter);
  unsigned hst = 0;
  if (e == cudaSuccess && iters)
    e = cudaMemcpyAsync(iters, dit, n_box * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, dst, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dev);
  free(hb);
  free(ho);
  free(hord);
  if (e != cudaSuccess) return SEA_ERR_CUDA;
  return (hst & SEA_FLAG_CG_CAP) ? SEA_ERR_CG_NOT_CONVERGED : SEA_OK;
}

sea_status sea_get_stats(const sea_ctx* c, sea_stats* s) {
  if (!c || !s) return SEA_ERR_ARG;
  *s = c->stats;
  s->n_launches = c->launches;
  // timings of the last sea_apply_ace, if its work has finished (no wait)
  if (c->apply_timed && cudaEventQuery(c->ev[8]) == cudaSuccess) {
    float t = 0;
    if (cudaEventElapsedTime(&t, c->ev[7], c->ev[8]) == cudaSuccess) s->ms_ace_apply = t;
    if (cudaEventElapsedTime(&t, c->ev[12], c->ev[13]) == cudaSuccess) s->ms_gram_apply = t;
    if (cudaEventElapsedTime(&t, c->ev[14], c->ev[15]) == cudaSuccess) s->ms_expand_apply = t;
  }
  cudaGetLastError();
  return SEA_OK;
}

const char* sea_last_error(const sea_ctx* c) {
  if (!c) return "NULL context";
  return c->err[0] ? c->err : "no error";
}

void sea_destroy(sea_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int k = 0; k < 2; ++k)
    if (c->xfer[k]) {
      cudaStreamSynchronize(c->xfer[k]);
      cudaStreamDestroy(c->xfer[k]);
    }
  for (cudaEvent_t e : c->xev)
    if (e) cudaEventDestroy(e);
  sea_batch_cache_free(c);
  for (LaunchGraph* g : {&c->g_chol, &c->g_plan})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  SeaBuf* all[] = {&c->phi, &c->vxx_dev, &c->psi_dev, &c->out_dev, &c->rowsum, &c->colsum,
                   &c->marg, &c->box, &c->cand_flag, &c->cand_geom, &c->list_a, &c->list_b,
                   &c->cand_S, &c->counts, &c->pinfo, &c->pS, &c->psize, &c->voff, &c->order,
                   &c->Q, &c->epair, &c->iters, &c->vbuf, &c->bbuf, &c->rbuf, &c->pbuf,
                   &c->qbuf, &c->eptr, &c->eent, &c->ewin, &c->coff, &c->cbuf, &c->status,
                   &c->exx_dev, &c->queue, &c->tmask, &c->tptr_o, &c->tlist_o, &c->tslot_o,
                   &c->tptr_t, &c->tlist_t, &c->partial, &c->Mbuf, &c->Abuf, &c->Lbuf, &c->wdig, &c->wx, &c->xevb, &c->gbuf, &c->flowbuf,
                   &c->scdm_u, &c->scdm_c,
                   &c->Linv, &c->Gbuf, &c->Hbuf, &c->Hbuf2, &c->bdesc, &c->bitems,
                   &c->onorm};
  for (SeaBuf* b : all) release(*b);
  for (int k = 0; k < 16; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  delete c;
}

}  // extern "C"
