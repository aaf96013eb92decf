// scdm.cu -- SCDM localization of canonical orbitals (Sec. II A).
//
//   Phi^T Pi = Q R               column-pivoted QR of the n x N matrix Phi^T
//                                (Eq. phi_qr); C = the first n pivots
//   B = (Phi^T)_{:,C}            n x n: B[j][k] = phi_j(r_{C_k})
//   X = Phi B,  P_CC = B^T B     (Eq. nonortho_scdm; X^T X dV = B^T B for
//                                orbitals orthonormal with the grid weight)
//   U = B P_CC^{-1/2},  Phi~ = Phi U   (Eqs. ortho_scdm, unitary_scdm)
//
// Only the pivot order of the QR is needed.  Column-pivoted QR picks, at
// step k, the column whose component orthogonal to the span of the k
// columns already chosen is longest; here that component's squared norm is
// kept for every grid point and downdated, c_r -= (q_k . a_r)^2, with q_k
// the unit vector of the new column after classical Gram-Schmidt against
// q_0..q_{k-1}, applied twice (the columns a_r of Phi^T have length n, so
// this work is small; the N-wide downdate is the cost).  Ties go to the
// smallest grid index.  P_CC^{-1/2} by the coupled Newton-Schulz iteration
// on P_CC / ||P_CC||_F (60 steps; the eigenvalues lie in (0, 1]).
#include "sea_internal.cuh"

namespace sea {
namespace {

// c[r] = sum_i phi[i][r]^2 (ascending i, fused multiply-add)
__global__ void k_scdm_norms(const double* __restrict__ phi, int n, size_t N,
                             double* __restrict__ c) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = phi[(size_t)i * N + r];
    s = fma(v, v, s);
  }
  c[r] = s;
}

// Per block: the largest c (ties: smallest index); selected points carry -1.
__global__ void __launch_bounds__(256)
    k_argmax1(const double* __restrict__ c, size_t N, double* __restrict__ bv,
              long long* __restrict__ bi) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double v = -2.0;
  long long idx = -1;
  for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (size_t)gridDim.x * blockDim.x)
    if (c[r] > v) {  // strict: keeps the first (smallest) index of this thread's stride
      v = c[r];
      idx = (long long)r;
    }
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double ov = sv[threadIdx.x + h];
      const long long oi = si[threadIdx.x + h];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi >= 0 && (si[threadIdx.x] < 0 || oi < si[threadIdx.x]))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bv[blockIdx.x] = sv[0];
    bi[blockIdx.x] = si[0];
  }
}

// Step k, one CTA: the pivot p = argmax over the block results; a = column
// p of Phi^T; two passes of classical Gram-Schmidt against Q[0..k); q_k =
// a / ||a|| into Q[k]; C[k] = p.
__global__ void __launch_bounds__(1024)
    k_scdm_pivot(const double* __restrict__ bv, const long long* __restrict__ bi, int nb,
                 const double* __restrict__ phi, int n, size_t N, int k, double* __restrict__ Q,
                 long long* __restrict__ C, double* __restrict__ work, unsigned* __restrict__ status) {
  __shared__ double sv[1024];
  __shared__ long long si[1024];
  double v = -2.0;
  long long idx = -1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (bv[b] > v || (bv[b] == v && bi[b] >= 0 && (idx < 0 || bi[b] < idx))) {
      v = bv[b];
      idx = bi[b];
    }
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double ov = sv[threadIdx.x + h];
      const long long oi = si[threadIdx.x + h];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi >= 0 && (si[threadIdx.x] < 0 || oi < si[threadIdx.x]))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const long long p = si[0];
  if (p < 0) {  // no point left: the orbitals are rank deficient
    if (threadIdx.x == 0) atomicOr(status, SEA_FLAG_NOT_PD);
    return;
  }
  double* a = work;          // [n]
  double* coef = work + n;   // [k]
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = phi[(size_t)i * N + p];
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s = fma(Q[(size_t)l * n + i], a[i], s);
      coef[l] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = a[i];
      for (int l = 0; l < k; ++l) s = fma(-coef[l], Q[(size_t)l * n + i], s);
      a[i] = s;
    }
    __syncthreads();
  }
  double nn = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) nn = fma(a[i], a[i], nn);
  __shared__ double red[1024];
  red[threadIdx.x] = nn;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
  if (!(red[0] > 0.0) && threadIdx.x == 0) atomicOr(status, SEA_FLAG_NOT_PD);
  for (int i = threadIdx.x; i < n; i += blockDim.x) Q[(size_t)k * n + i] = a[i] * inv;
  if (threadIdx.x == 0) C[k] = p;
}

// c[r] -= (q_k . a_r)^2 for every grid point; the pivot is marked -1.
__global__ void k_scdm_downdate(const double* __restrict__ phi, int n, size_t N,
                                const double* __restrict__ q, const long long* __restrict__ Ck,
                                double* __restrict__ c) {
  extern __shared__ double sq[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) sq[i] = q[i];
  __syncthreads();
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  if ((long long)r == *Ck) {
    c[r] = -1.0;
    return;
  }
  if (c[r] < 0.0) return;
  double d = 0.0;
  for (int i = 0; i < n; ++i) d = fma(sq[i], phi[(size_t)i * N + r], d);
  c[r] = fma(-d, d, c[r]);
}

// B[j][k] = phi[j][C[k]]
__global__ void k_scdm_gather(const double* __restrict__ phi, int n, size_t N,
                              const long long* __restrict__ C, double* __restrict__ B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int j = t / n, k = t % n;
  B[t] = phi[(size_t)j * N + C[k]];
}

// C = alpha op(A) op(B) + beta C for n x n matrices (row-major), op = T if
// the flag is set.  16 x 16 tiles.
__global__ void k_gemm_nn(const double* __restrict__ A, int ta, const double* __restrict__ Bm,
                          int tb, int n, double alpha, double beta, double* __restrict__ Cm) {
  __shared__ double As[16][17], Bs[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] =
        (i < n && ka < n) ? (ta ? A[(size_t)ka * n + i] : A[(size_t)i * n + ka]) : 0.0;
    Bs[threadIdx.y][threadIdx.x] =
        (kb < n && j < n) ? (tb ? Bm[(size_t)j * n + kb] : Bm[(size_t)kb * n + j]) : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (i < n && j < n) Cm[(size_t)i * n + j] = alpha * acc + (beta != 0.0 ? beta * Cm[(size_t)i * n + j] : 0.0);
}

// s = ||P||_F (one CTA, fixed order)
__global__ void __launch_bounds__(1024) k_frob(const double* __restrict__ P, int n2, double* __restrict__ s) {
  __shared__ double red[1024];
  double v = 0.0;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) v = fma(P[t], P[t], v);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *s = sqrt(red[0]);
}

// Y = P / s, Z = I
__global__ void k_ns_init(const double* __restrict__ P, int n, const double* __restrict__ s,
                          double* __restrict__ Y, double* __restrict__ Z) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  Y[t] = P[t] / *s;
  Z[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// T = (3 I - T) / 2 in place (T holds Z Y)
__global__ void k_ns_t(double* __restrict__ T, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  T[t] = 0.5 * (((t / n == t % n) ? 3.0 : 0.0) - T[t]);
}

// Z /= sqrt(s)
__global__ void k_ns_scale(double* __restrict__ Z, int n, const double* __restrict__ s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) Z[t] /= sqrt(*s);
}

// out[i][r] = sum_j U[j][i] phi[j][r]: thread per point r, U in shared memory
// in chunks of 32 columns i.
__global__ void __launch_bounds__(256)
    k_rotate(const double* __restrict__ phi, int n, size_t N, const double* __restrict__ U,
             double* __restrict__ out) {
  __shared__ double su[64][33];
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int i0 = 0; i0 < n; i0 += 32) {
    double acc[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u] = 0.0;
    for (int j0 = 0; j0 < n; j0 += 64) {
      __syncthreads();
      for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
        const int jj = q / 32, ii = q % 32;
        su[jj][ii] = (j0 + jj < n && i0 + ii < n) ? U[(size_t)(j0 + jj) * n + i0 + ii] : 0.0;
      }
      __syncthreads();
      if (r < N)
        for (int jj = 0; jj < 64 && j0 + jj < n; ++jj) {
          const double v = phi[(size_t)(j0 + jj) * N + r];
#pragma unroll
          for (int u = 0; u < 32; ++u) acc[u] = fma(su[jj][u], v, acc[u]);
        }
    }
    if (r < N)
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (i0 + u < n) out[(size_t)(i0 + u) * N + r] = acc[u];
  }
}

}  // namespace

// SCDM on the orbitals in c->phi (n_orb x ng): U (device, n x n) and the
// pivots C (device, n); the localized orbitals replace c->phi (through
// c->vxx_dev as scratch).
cudaError_t launch_scdm(sea_ctx* c, double* U_dev, long long* C_dev) {
  const int n = c->n_orb;
  const size_t N = c->ng;
  const int nb = 1024;  // blocks of the first argmax stage
  if (!sea_ensure(c, c->cand_S, std::max<size_t>(N * sizeof(double), 64)) ||
      !sea_ensure(c, c->Mbuf, (size_t)n * n * sizeof(double)) ||   // Q (rows q_k)
      !sea_ensure(c, c->Lbuf, (size_t)n * n * sizeof(double)) ||   // B
      !sea_ensure(c, c->Linv, (size_t)n * n * sizeof(double)) ||   // P_CC, then T
      !sea_ensure(c, c->Gbuf, (size_t)n * n * sizeof(double)) ||   // Y
      !sea_ensure(c, c->Hbuf, (size_t)n * n * sizeof(double)) ||   // Z
      !sea_ensure(c, c->Hbuf2, (size_t)n * n * sizeof(double)) ||  // scratch
      !sea_ensure(c, c->Abuf, (size_t)(2 * n + 4 * nb + 8) * sizeof(double)))
    return cudaErrorMemoryAllocation;
  const double* phi = (const double*)c->phi.p;
  double* cn = (double*)c->cand_S.p;
  double* Q = (double*)c->Mbuf.p;
  double* B = (double*)c->Lbuf.p;
  double* P = (double*)c->Linv.p;
  double* Y = (double*)c->Gbuf.p;
  double* Z = (double*)c->Hbuf.p;
  double* T = (double*)c->Hbuf2.p;
  double* work = (double*)c->Abuf.p;        // [n] + [n]
  double* bv = work + 2 * n;                 // [nb]
  long long* bi = (long long*)(bv + nb);     // [nb]
  double* sF = bv + 3 * nb;                  // scalar
  unsigned* status = (unsigned*)c->status.p;
  cudaStream_t st = c->stream;
  const unsigned gN = (unsigned)((N + 255) / 256);
  k_scdm_norms<<<gN, 256, 0, st>>>(phi, n, N, cn);
  for (int k = 0; k < n; ++k) {
    k_argmax1<<<nb, 256, 0, st>>>(cn, N, bv, bi);
    k_scdm_pivot<<<1, 1024, 0, st>>>(bv, bi, nb, phi, n, N, k, Q, C_dev, work, status);
    k_scdm_downdate<<<gN, 256, (size_t)n * sizeof(double), st>>>(phi, n, N, Q + (size_t)k * n,
                                                                  C_dev + k, cn);
  }
  const unsigned gnn = (unsigned)((n * n + 255) / 256);
  const dim3 gg((n + 15) / 16, (n + 15) / 16), tb(16, 16);
  k_scdm_gather<<<gnn, 256, 0, st>>>(phi, n, N, C_dev, B);
  k_gemm_nn<<<gg, tb, 0, st>>>(B, 1, B, 0, n, 1.0, 0.0, P);  // P = B^T B
  k_frob<<<1, 1024, 0, st>>>(P, n * n, sF);
  k_ns_init<<<gnn, 256, 0, st>>>(P, n, sF, Y, Z);
  for (int it = 0; it < 60; ++it) {
    k_gemm_nn<<<gg, tb, 0, st>>>(Z, 0, Y, 0, n, 1.0, 0.0, T);  // T = Z Y
    k_ns_t<<<gnn, 256, 0, st>>>(T, n);                         // T = (3I - Z Y)/2
    k_gemm_nn<<<gg, tb, 0, st>>>(Y, 0, T, 0, n, 1.0, 0.0, P);  // Y T (P as scratch)
    cudaMemcpyAsync(Y, P, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    k_gemm_nn<<<gg, tb, 0, st>>>(T, 0, Z, 0, n, 1.0, 0.0, P);  // T Z
    cudaMemcpyAsync(Z, P, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  k_ns_scale<<<gnn, 256, 0, st>>>(Z, n, sF);                 // P_CC^{-1/2}
  k_gemm_nn<<<gg, tb, 0, st>>>(B, 0, Z, 0, n, 1.0, 0.0, U_dev);  // U = B P^{-1/2}
  double* out = (double*)c->vxx_dev.p;
  k_rotate<<<gN, 256, 0, st>>>(phi, n, N, U_dev, out);
  cudaMemcpyAsync(c->phi.p, out, (size_t)n * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  c->launches += 1 + 3 * n + 4 + 60 * 4 + 3;
  return cudaGetLastError();
}

}  // namespace sea
