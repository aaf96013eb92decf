// accum.cu -- far field and deterministic accumulation of D (Eq. tDxx),
// V_xx phi = -D (Eq. DxxVxx) and E_xx (Eq. exxGen_mlwf).
//
// Every selected pair p = (i, j) makes one or two entries:
//   orbital i receives v_ij phi_j on Omega^D_ij (Omega_jj if j != i,
//   scale_2x Omega_ii if j == i), and for j != i orbital j receives
//   v_ij phi_i on Omega_ii (v_ji = v_ij).
// v_ij is the CG solution inside Omega_ij and the multipole expansion
// (Eq. me) outside it.
//   k_contrib   (grid over entries x chunks): c = v * phi_partner on the
//               entry's window, stored per entry; no accumulation here.
//   k_accumulate (CTA per orbital x z-plane): the plane is built in
//               shared memory from zero, each entry of the orbital
//               subtracted in pair order (a fixed order: no floating-point
//               atomics), then stored once to the output and, when given,
//               to a second output (the caller's copy; the context's copy
//               is then stored only on the tiles the orbital's windows
//               touch).  Planes too large for shared memory take the same
//               steps on a global slab, with full stores.
#include <algorithm>

#include "sea_internal.cuh"

namespace sea {

// Window of orbital o's box [s, s+L) for a pair whose domain is [lo, lo+ext)
// on an axis of n points: the box shifted by kshift*n, or, for a box that
// spans the whole axis, the n-point window centred on the pair domain.
__device__ __forceinline__ void box_window(int s, int L, int kshift, int n, int lo, int ext,
                                           int* ws, int* wl) {
  if (L >= n) {
    *ws = lo - (n - ext) / 2;
    *wl = n;
  } else {
    *ws = s + kshift * n;
    *wl = L;
  }
}

// scale_2x: the extent doubled about the interval centre, rounded outward
// (even L: [s - L/2, s + 3L/2); odd L: [c - L, c + L] with c = s + (L-1)/2),
// capped at n points centred on the interval (ties low).
__device__ __forceinline__ void scale_twice(int s, int L, int n, int* ws, int* wl) {
  int lo2, len2;
  if ((L & 1) == 0) {
    lo2 = s - L / 2;
    len2 = 2 * L;
  } else {
    lo2 = s + (L - 1) / 2 - L;
    len2 = 2 * L + 1;
  }
  if (len2 >= n) {
    lo2 += (len2 - n) / 2;
    len2 = n;
  }
  *ws = lo2;
  *wl = len2;
}

// Thread per orbital: count (mode 0) or write (mode 1) its entries in pair
// order.  eptr must hold the exclusive scan of the counts for mode 1.
// Warp per orbital: the lanes test 32 pairs at a time and the entries of o
// are numbered in pair order by ballots (deterministic).
__global__ void k_entries(const PairInfo* __restrict__ pinfo, const int* __restrict__ npairs,
                          const int* __restrict__ box, int n_orb, int nx, int ny, int nz,
                          int mode, int* __restrict__ ecount, const int* __restrict__ eptr,
                          Entry* __restrict__ ent) {
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (o >= n_orb) return;  // warp-uniform
  const int P = *npairs;
  const int N[3] = {nx, ny, nz};
  int cnt = 0;
  int pos = mode ? eptr[o] : 0;
  for (int p0 = 0; p0 < P; p0 += 32) {
    const int p = p0 + lane;
    int role = -1;
    int pi = -1, pj = -1;
    if (p < P) {
      pi = pinfo[p].i;
      pj = pinfo[p].j;
      role = pi == o ? 0 : (pj == o ? 1 : -1);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, role >= 0);
    if (mode && role >= 0) {
      const PairInfo I = pinfo[p];
      Entry e;
      e.pair = p;
      e.o = o;
      e.partner = role == 0 ? I.j : I.i;
      for (int a = 0; a < 3; ++a) {
        if (role == 0 && I.i == I.j) {
          int s0, l0;
          box_window(box[I.i * 6 + a], box[I.i * 6 + 3 + a], 0, N[a], I.lo[a], I.ext[a], &s0, &l0);
          scale_twice(s0, l0, N[a], &e.ws[a], &e.wl[a]);
        } else if (role == 0) {
          box_window(box[I.j * 6 + a], box[I.j * 6 + 3 + a], I.k[a], N[a], I.lo[a], I.ext[a],
                     &e.ws[a], &e.wl[a]);
        } else {
          box_window(box[I.i * 6 + a], box[I.i * 6 + 3 + a], 0, N[a], I.lo[a], I.ext[a], &e.ws[a],
                     &e.wl[a]);
        }
      }
      ent[pos + __popc(mask & ((1u << lane) - 1u))] = e;
    }
    pos += __popc(mask);
    cnt += __popc(mask);
  }
  if (!mode && lane == 0) ecount[o] = cnt;
}

// Single-CTA exclusive scan of n ints (n small); total into *tot.
__global__ void k_scan_int(const int* __restrict__ in, int n, int* __restrict__ out,
                           int* __restrict__ tot) {
  __shared__ long long part[32];
  const int T = blockDim.x, chunk = (n + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(n, b + chunk);
  long long s = 0;
  for (int x = b; x < e; ++x) s += in[x];
  long long acc = 0;
  long long pos = block_exscan_ll(s, part, &acc);
  if (threadIdx.x == 0) *tot = (int)acc;
  for (int x = b; x < e; ++x) {
    out[x] = (int)pos;
    pos += in[x];
  }
  if (threadIdx.x == T - 1) out[n] = (int)pos;
}

// Window sizes of all entries, then their exclusive scan (64-bit).
__global__ void k_entry_offsets(const Entry* __restrict__ ent, const int* __restrict__ E_dev,
                                long long* __restrict__ coff, long long* __restrict__ tot,
                                long long* __restrict__ maxwin) {
  __shared__ long long part[32];
  const int E = *E_dev;
  const int T = blockDim.x, chunk = (E + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(E, b + chunk);
  long long s = 0, mx = 0;
  for (int x = b; x < e; ++x) {
    const long long w = (long long)ent[x].wl[0] * ent[x].wl[1] * ent[x].wl[2];
    s += w;
    mx = w > mx ? w : mx;
  }
  long long acc = 0;
  long long pos = block_exscan_ll(s, part, &acc);
  const long long m = block_max_ll(mx, part);
  if (threadIdx.x == 0) {
    *tot = acc;
    *maxwin = m;
  }
  for (int x = b; x < e; ++x) {
    coff[x] = pos;
    pos += (long long)ent[x].wl[0] * ent[x].wl[1] * ent[x].wl[2];
  }
}

// Window contributions of the entries (grid y) in chunks of SEA_CHUNK window
// points (grid x); `part` as in contrib_range (1: the far field on a side
// stream beside the CG, 2: the points inside the pair boxes after it).  DFM: double-float arithmetic (mixed form),
// four CTAs per SM there (64 registers, no spills): the nested Horner steps
// of the potential are one dependent chain per point, so the warps resident
// per SM set the rate (measured 0.81 -> 0.77 ms per step against two CTAs).
template <bool DFM>
__global__ void __launch_bounds__(256, DFM ? 4 : 1)
    k_contrib(const double* __restrict__ phi, int nx, int ny, int nz, const Entry* __restrict__ ent,
              const long long* __restrict__ coff, const PairInfo* __restrict__ pinfo,
              const long long* __restrict__ voff, const double* __restrict__ vbuf,
              const double* __restrict__ Qg, double hx, double hy, double hz,
              double* __restrict__ cbuf, int part) {
  const Entry e = ent[blockIdx.y];
  const PairInfo P = pinfo[e.pair];
  const int nw = e.wl[0] * e.wl[1] * e.wl[2];
  const WinSplit sp = window_split(e, P);
  // parts 1 and 2 enumerate their own points (divisions exact below 2^24)
  const bool compact = part != 0 && nw < (1 << 24);
  const int cnt = !compact ? nw : part == 1 ? sp.n_out : sp.n_in;
  const int t0 = blockIdx.x * SEA_CHUNK;
  if (t0 >= cnt) return;
  __shared__ double Ps[SEA_NMONO];
  __shared__ DF Pd[SEA_NMONO];
  if (part != 2 && threadIdx.x < SEA_NMONO) {
    const double q = Qg[(size_t)e.pair * SEA_QSTRIDE + SEA_NQ + threadIdx.x];
    if (DFM)
      Pd[threadIdx.x] = df_from_double(q);
    else
      Ps[threadIdx.x] = q;
  }
  __syncthreads();
  contrib_range<DFM>(part, compact, sp, e, P, phi, nx, ny, nz, vbuf + voff[e.pair], Pd, Ps, hx, hy,
                     hz, cbuf + coff[blockIdx.y], t0, min(cnt, t0 + SEA_CHUNK));
}

// Global-memory form: CTA per (orbital, slab of SLAB z-planes); out2, when
// given, receives the finished slab.
#define SEA_SLAB 4
// Largest plane (bytes) built in shared memory.
#define SEA_ACC_SMEM_MAX (200 * 1024)
__global__ void __launch_bounds__(256)
    k_accumulate_gmem(int nx, int ny, int nz, int o_begin, const int* __restrict__ eptr,
                      const Entry* __restrict__ ent, const long long* __restrict__ coff,
                      const double* __restrict__ cbuf, double* __restrict__ out,
                      double* __restrict__ out2) {
  const int o = o_begin + blockIdx.x;
  const int z0 = blockIdx.y * SEA_SLAB, z1 = min(nz, z0 + SEA_SLAB);
  const size_t plane = (size_t)nx * ny;
  double* Do = out + (size_t)o * plane * nz;
  for (size_t g = z0 * plane + threadIdx.x; g < (size_t)z1 * plane; g += blockDim.x) Do[g] = 0.0;
  const int e0 = eptr[o], e1 = eptr[o + 1];
  for (int k = e0; k < e1; ++k) {
    __syncthreads();
    const Entry e = ent[k];
    const double* c = cbuf + coff[k];
    const int wx = e.wl[0], wy = e.wl[1];
    const int rowpts = wx * wy;
    for (int tz = 0; tz < e.wl[2]; ++tz) {
      const int gz = wrapi(e.ws[2] + tz, nz);
      if (gz < z0 || gz >= z1) continue;
      for (int r = threadIdx.x; r < rowpts; r += blockDim.x) {
        const int tx = r % wx, ty = r / wx;
        const size_t g = ((size_t)gz * ny + wrapi(e.ws[1] + ty, ny)) * nx + wrapi(e.ws[0] + tx, nx);
        Do[g] = __dsub_rn(Do[g], c[(size_t)tz * rowpts + r]);
      }
    }
  }
  if (out2) {
    __syncthreads();
    double* D2 = out2 + (size_t)o * plane * nz;
    for (size_t g = z0 * plane + threadIdx.x; g < (size_t)z1 * plane; g += blockDim.x) D2[g] = Do[g];
  }
}

// Cyclic window [s, s + L) (s in [0, n)) meets [a, b) (0 <= a < b <= n).
__device__ __forceinline__ bool cyc_hits(int s, int L, int a, int b, int n) {
  if (L >= n) return true;
  if (max(a, s) < min(b, s + L)) return true;
  return a < min(b, s + L - n);  // the wrapped part [0, s + L - n)
}

// Shared-memory form: CTA per (orbital, z-plane), the plane (nx*ny
// doubles) in dynamic shared memory.  A thread walks the window rows of an
// entry with its (tx, ty) advanced by the CTA stride, without divisions.
// With a second output (the caller's copy, written in full), the context's
// copy is stored only on the tiles (TX x TY x TZ) that a window of the
// orbital touches: the tiles of the orbital's W lists, the only places the
// ACE kernels read it (tile mask after the plane, in shared memory).
#define SEA_ACC_MAXE 64
#define SEA_ACC_THREADS 512
__global__ void __launch_bounds__(SEA_ACC_THREADS)
    k_accumulate(int nx, int ny, int nz, int o_begin, const int* __restrict__ eptr,
                 const Entry* __restrict__ ent, const long long* __restrict__ coff,
                 const double* __restrict__ cbuf, double* __restrict__ out,
                 double* __restrict__ out2, int bulk) {
  extern __shared__ double sp[];
  __shared__ int es[SEA_ACC_MAXE][5];  // x start, x length, y start, y length, meets the z tile
  const int o = o_begin + blockIdx.x;
  const int z = blockIdx.y;
  const int plane = nx * ny;
  unsigned char* tmask = reinterpret_cast<unsigned char*>(sp + plane);
  if ((plane & 1) == 0) {
    double2* sp2 = reinterpret_cast<double2*>(sp);
    for (int g = threadIdx.x; g < plane / 2; g += blockDim.x) sp2[g] = make_double2(0.0, 0.0);
  } else {
    for (int g = threadIdx.x; g < plane; g += blockDim.x) sp[g] = 0.0;
  }
  const int e0 = eptr[o], e1 = eptr[o + 1];
  for (int k = e0; k < e1; ++k) {
    const Entry e = ent[k];
    const int tz = wrapi(z - e.ws[2], nz);
    if (tz >= e.wl[2]) continue;  // uniform over the CTA
    __syncthreads();
    const int wx = e.wl[0], wy = e.wl[1];
    const int rowpts = wx * wy;
    const double* c = cbuf + coff[k] + (size_t)tz * rowpts;
    const int x0 = wrapi(e.ws[0], nx), y0 = wrapi(e.ws[1], ny);
    const int sy = blockDim.x / wx, sx = blockDim.x - sy * wx;  // stride as (rows, columns)
    int ty = threadIdx.x / wx, tx = threadIdx.x - ty * wx;
    for (int r = threadIdx.x; r < rowpts; r += blockDim.x) {
      int gx = x0 + tx, gy = y0 + ty;
      gx -= gx >= nx ? nx : 0;
      gy -= gy >= ny ? ny : 0;
      const int g = gy * nx + gx;
      sp[g] = __dsub_rn(sp[g], c[r]);
      tx += sx;
      ty += sy;
      if (tx >= wx) {
        tx -= wx;
        ++ty;
      }
    }
  }
  const int ntx = (nx + TX - 1) / TX;
  const bool all = out2 == nullptr || e1 - e0 > SEA_ACC_MAXE;  // uniform
  if (!all) {
    const int t = threadIdx.x;
    if (t < e1 - e0) {
      const Entry e = ent[e0 + t];
      const int zs = (z / TZ) * TZ;
      es[t][0] = wrapi(e.ws[0], nx);
      es[t][1] = e.wl[0];
      es[t][2] = wrapi(e.ws[1], ny);
      es[t][3] = e.wl[1];
      es[t][4] = cyc_hits(wrapi(e.ws[2], nz), e.wl[2], zs, min(nz, zs + TZ), nz);
    }
    __syncthreads();
    const int nty = (ny + TY - 1) / TY;
    for (int q = threadIdx.x; q < ntx * nty; q += blockDim.x) {
      const int qy = q / ntx, qx = q - qy * ntx;
      const int ax = qx * TX, bx = min(nx, ax + TX), ay = qy * TY, by = min(ny, ay + TY);
      bool hit = false;
      for (int k = 0; k < e1 - e0; ++k)
        hit = hit || (es[k][4] && cyc_hits(es[k][0], es[k][1], ax, bx, nx) &&
                      cyc_hits(es[k][2], es[k][3], ay, by, ny));
      tmask[q] = hit ? 1 : 0;
    }
  }
  const size_t base = ((size_t)o * nz + z) * plane;
  // The output stored in full (out2, else out when every tile is wanted) by
  // one bulk copy of the plane from shared memory when `bulk` (the plane is
  // a multiple of 16 bytes and the outputs 16-byte aligned): the generic
  // writes are made visible to the copy engine, then thread 0 issues it and
  // waits, before the CTA ends, until the plane has been read.
  double* full = out2 ? out2 : (all ? out : nullptr);
  const bool by_copy = bulk && full != nullptr;
  if (by_copy) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (by_copy && threadIdx.x == 0) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(full + base),
                 "r"((uint32_t)__cvta_generic_to_shared(sp)), "r"((uint32_t)plane * 8u)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  const int nty = (ny + TY - 1) / TY;
  if (by_copy && out2 != nullptr && !all) {
    // the context's copy on the marked tiles only: a thread per tile, its
    // rows as 16-byte pieces when rows and outputs allow it
    const bool v2 = (nx & 1) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    for (int q = threadIdx.x; q < ntx * nty; q += blockDim.x) {
      if (!tmask[q]) continue;
      const int qy = q / ntx, qx = q - qy * ntx;
      const int x0 = qx * TX, x1 = min(nx, x0 + TX), y1 = min(ny, qy * TY + TY);
      for (int y = qy * TY; y < y1; ++y) {
        const int g0 = y * nx;
        if (v2) {
          for (int x = x0; x < x1; x += 2)
            *reinterpret_cast<double2*>(out + base + g0 + x) =
                *reinterpret_cast<const double2*>(sp + g0 + x);
        } else {
          for (int x = x0; x < x1; ++x) out[base + g0 + x] = sp[g0 + x];
        }
      }
    }
  } else if (!(by_copy && out2 == nullptr)) {  // else the copy stored everything
    const int dy = blockDim.x / nx, dx = blockDim.x - dy * nx;  // (x, y) of g, without divisions
    int y = threadIdx.x / nx, x = threadIdx.x - y * nx;
    for (int g = threadIdx.x; g < plane; g += blockDim.x) {
      const double v = sp[g];
      if (out2 && !by_copy) out2[base + g] = v;
      if (all || tmask[(y / TY) * ntx + x / TX]) out[base + g] = v;
      x += dx;
      y += dy;
      if (x >= nx) {
        x -= nx;
        ++y;
      }
    }
  }
  if (by_copy && threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// E_xx = -sum_p (2 - delta_ij) e_p in pair order, plus CG statistics:
// res[0] = E_xx, res[1] = sum |Omega_ij| x iterations, res[2..4] = min,
// max, mean iterations.
__global__ void __launch_bounds__(256) k_exx(const PairInfo* __restrict__ pinfo,
                                              const int* __restrict__ npairs,
                                              const double* __restrict__ epair,
                                              const int* __restrict__ iters,
                                              double* __restrict__ res) {
  // thread t sums a contiguous range of pairs in order, then the block sums
  // the threads' values in a fixed order (deterministic)
  __shared__ double red[3][32];
  __shared__ int ired[2][32];
  const int P = *npairs;
  const int T = blockDim.x, chunk = (P + T - 1) / T;
  const int p0 = threadIdx.x * chunk, p1 = min(P, p0 + chunk);
  double e = 0.0, ui = 0.0, sum = 0.0;
  int mn = 0x7fffffff, mx = 0;
  for (int p = p0; p < p1; ++p) {
    const PairInfo I = pinfo[p];
    e += (I.i == I.j ? 1.0 : 2.0) * epair[p];
    const int it = iters[p] < 0 ? -iters[p] : iters[p];
    ui += (double)I.n * it;
    sum += it;
    mn = min(mn, it);
    mx = max(mx, it);
  }
  e = block_sum(e, red[0]);
  ui = block_sum(ui, red[1]);
  sum = block_sum(sum, red[2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    ired[0][threadIdx.x >> 5] = mn;
    ired[1][threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (T >> 5); ++k) {
      mn = min(mn, ired[0][k]);
      mx = max(mx, ired[1][k]);
    }
    mn = min(mn, ired[0][0]);
    mx = max(mx, ired[1][0]);
    res[0] = -e;
    res[1] = ui;
    res[2] = P ? mn : 0;
    res[3] = mx;
    res[4] = P ? sum / P : 0.0;
  }
}

cudaError_t launch_entries(sea_ctx* c) {
  const int n = c->n_orb;
  int* counts = (int*)c->counts.p;
  k_entries<<<(n + 7) / 8, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p, counts + 1,
                                                (const int*)c->box.p, n, c->N[0], c->N[1],
                                                c->N[2], 0, (int*)c->eent.p, nullptr, nullptr);
  // counts were written into the start of eent as scratch: scan them into eptr
  k_scan_int<<<1, 1024, 0, c->stream>>>((const int*)c->eent.p, n, (int*)c->eptr.p, counts + 2);
  k_entries<<<(n + 7) / 8, 256, 0, c->stream>>>((const PairInfo*)c->pinfo.p, counts + 1,
                                                (const int*)c->box.p, n, c->N[0], c->N[1],
                                                c->N[2], 1, nullptr, (const int*)c->eptr.p,
                                                (Entry*)c->ewin.p);
  k_entry_offsets<<<1, 1024, 0, c->stream>>>((const Entry*)c->ewin.p, counts + 2,
                                             (long long*)c->coff.p, (long long*)(counts + 6),
                                             (long long*)(counts + 8));
  c->launches += 4;
  return cudaGetLastError();
}

// Window contributions and their accumulation for orbitals [o_begin, o_end),
// whose entries are [e_begin, e_end) (entries are grouped by orbital).
cudaError_t launch_accumulate_range(sea_ctx* c, double* out, int o_begin, int o_end, int e_begin,
                                    int e_end, double* out2) {
  if (e_end > e_begin) {
    const int chunks = (int)((c->max_window + SEA_CHUNK - 1) / SEA_CHUNK);
    for (int e0 = e_begin; e0 < e_end; e0 += 65535) {
      const int ne = std::min(65535, e_end - e0);
      auto kern = c->prm.precision == 1 ? k_contrib<true> : k_contrib<false>;
      kern<<<dim3(chunks, ne), 256, 0, c->stream>>>(
          (const double*)c->phi.p, c->N[0], c->N[1], c->N[2], (const Entry*)c->ewin.p + e0,
          (const long long*)c->coff.p + e0, (const PairInfo*)c->pinfo.p,
          (const long long*)c->voff.p, (const double*)c->vbuf.p, (const double*)c->Q.p, c->h[0],
          c->h[1], c->h[2], (double*)c->cbuf.p, c->far_side ? 2 : 0);
      c->launches += 1;
    }
  }
  if (o_end > o_begin) {
    if (c->far_side) {  // the contributions outside the pair boxes are in
      const cudaError_t e = cudaStreamWaitEvent(c->stream, c->xev[1], 0);
      if (e != cudaSuccess) return e;
    }
    // the plane, then one tile-mask byte per (x tile, y tile)
    const size_t smem = (size_t)c->N[0] * c->N[1] * sizeof(double) +
                        (size_t)((c->N[0] + TX - 1) / TX) * ((c->N[1] + TY - 1) / TY);
    if (smem <= SEA_ACC_SMEM_MAX) {
      cudaError_t e = cudaFuncSetAttribute(k_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
      // bulk plane copies: whole planes of 16-byte multiples into 16-byte
      // aligned outputs
      const bool plane16 = ((size_t)c->N[0] * c->N[1] * sizeof(double)) % 16 == 0;
      const bool al16 = ((uintptr_t)out % 16 == 0) && ((uintptr_t)out2 % 16 == 0);
      k_accumulate<<<dim3(o_end - o_begin, c->N[2]), SEA_ACC_THREADS, smem, c->stream>>>(
          c->N[0], c->N[1], c->N[2], o_begin, (const int*)c->eptr.p, (const Entry*)c->ewin.p,
          (const long long*)c->coff.p, (const double*)c->cbuf.p, out, out2,
          plane16 && al16 ? 1 : 0);
    } else {
      k_accumulate_gmem<<<dim3(o_end - o_begin, (c->N[2] + SEA_SLAB - 1) / SEA_SLAB), 256, 0,
                          c->stream>>>(c->N[0], c->N[1], c->N[2], o_begin, (const int*)c->eptr.p,
                                       (const Entry*)c->ewin.p, (const long long*)c->coff.p,
                                       (const double*)c->cbuf.p, out, out2);
    }
    c->launches += 1;
  }
  return cudaGetLastError();
}

// The contributions outside each pair box (they need the moments alone) on
// the context's first copy stream, beside the CG: submitted after the CG's
// launch, whose persistent CTAs fill the GPU, they take the SMs that the CG's
// last pairs leave idle.  The accumulation later forms the points inside
// the boxes and waits for this launch.  Mixed form only.
cudaError_t launch_contrib_far(sea_ctx* c, cudaEvent_t setup_done) {
  c->far_side = false;
  if (c->prm.precision != 1 || c->E == 0) return cudaSuccess;
  cudaError_t e = cudaStreamWaitEvent(c->xfer[0], setup_done, 0);
  if (e != cudaSuccess) return e;
  const int chunks = (int)((c->max_window + SEA_CHUNK - 1) / SEA_CHUNK);
  for (int e0 = 0; e0 < c->E; e0 += 65535) {
    const int ne = std::min(65535, c->E - e0);
    k_contrib<true><<<dim3(chunks, ne), 256, 0, c->xfer[0]>>>(
        (const double*)c->phi.p, c->N[0], c->N[1], c->N[2], (const Entry*)c->ewin.p + e0,
        (const long long*)c->coff.p + e0, (const PairInfo*)c->pinfo.p,
        (const long long*)c->voff.p, (const double*)c->vbuf.p, (const double*)c->Q.p, c->h[0],
        c->h[1], c->h[2], (double*)c->cbuf.p, 1);
    c->launches += 1;
  }
  e = cudaEventRecord(c->xev[1], c->xfer[0]);
  if (e != cudaSuccess) return e;
  c->far_side = true;
  return cudaGetLastError();
}

// E_xx and the CG statistics (after every pair energy is final), on
// stream st.
cudaError_t launch_exx(sea_ctx* c, cudaStream_t st) {
  k_exx<<<1, 256, 0, st>>>((const PairInfo*)c->pinfo.p, (const int*)c->counts.p + 1,
                                 (const double*)c->epair.p, (const int*)c->iters.p,
                                 (double*)c->exx_dev.p);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_accumulate(sea_ctx* c, double* out, double* out2, bool with_exx) {
  cudaError_t e = launch_accumulate_range(c, out, 0, c->n_orb, 0, c->E, out2);
  return e != cudaSuccess || !with_exx ? e : launch_exx(c, c->stream);
}

cudaError_t upload_harmonics_accum() { return upload_harmonics_here(); }

}  // namespace sea
