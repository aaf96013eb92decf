// noalloc.cu -- sea_poisson_batch_noalloc: the batched box Poisson solver
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: plugins whose host framework owns
// all device memory through its own pool (a call to cudaMalloc behind its
// back breaks its accounting or fails outright), and processes whose device
// footprint is fixed at start-up and must not grow afterwards.  For them
// this entry point runs the same CG kernel as sea_poisson_batch, but its
// scratch (CG vectors r, p, q, the box records, offsets, order, iteration
// counts, status word and work-queue counter) lives in one file-scope
// __device__ array of fixed size instead of memory allocated per call.
//
// Costs and limits: every GPU that loads this library holds the array
// (about 25 MB) until the process exits.  At most SEA_NOALLOC_MAX_BOXES
// boxes and SEA_NOALLOC_MAX_UNKNOWNS unknowns per call; larger requests are
// rejected with SEA_ERR_LIMIT before any GPU work.  All calls share the one
// array: calls that overlap on the GPU (different streams, or threads of
// one process, without ordering between them) race and corrupt each
// other's scratch; order them.  The array keeps the previous call's
// contents, so every value that must start at zero (status word, queue
// counter) is cleared by each call.
//
// The call is synchronous: it copies the box extents in and the iteration
// counts and status out through pageable host memory and waits for the
// stream.  It must therefore not be made while its stream is being captured
// into a CUDA graph; a capturing stream is detected first and the call
// returns SEA_ERR_ARG before it queues anything, so the caller's capture
// stays valid.
//
// The array's device address is looked up once per device, on the first
// call made with that device current (cudaGetSymbolAddress).
#include <mutex>

#include "sea_internal.cuh"

#define SEA_NOALLOC_MAX_BOXES 4096
#define SEA_NOALLOC_MAX_UNKNOWNS (1 << 20)
#define SEA_NOALLOC_MAX_DEVICES 64

namespace {

// Layout of the scratch, in bytes from the start of the array.
constexpr size_t kVec = (size_t)SEA_NOALLOC_MAX_UNKNOWNS * sizeof(double);
constexpr size_t kOffR = 0;
constexpr size_t kOffP = kOffR + kVec;
constexpr size_t kOffQ = kOffP + kVec;
constexpr size_t kOffBox = kOffQ + kVec;
constexpr size_t kOffVoff = kOffBox + (size_t)SEA_NOALLOC_MAX_BOXES * sizeof(PairInfo);
constexpr size_t kOffOrder = kOffVoff + (size_t)SEA_NOALLOC_MAX_BOXES * sizeof(long long);
constexpr size_t kOffIters = kOffOrder + (size_t)SEA_NOALLOC_MAX_BOXES * sizeof(int);
constexpr size_t kOffExt = kOffIters + (size_t)SEA_NOALLOC_MAX_BOXES * sizeof(int);
constexpr size_t kOffMisc = kOffExt + (size_t)SEA_NOALLOC_MAX_BOXES * 3 * sizeof(int);
constexpr size_t kMiscBytes = 256;  // status word, queue counter
constexpr size_t kScratchBytes = kOffMisc + kMiscBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[SEA_NOALLOC_MAX_DEVICES] = {};

// Box records from the extents: sizes and exclusive-scan offsets.  One
// CTA; each thread scans a contiguous chunk.
__global__ void k_noalloc_records(const int* __restrict__ ext, int nbox,
                                  PairInfo* __restrict__ boxes, long long* __restrict__ voff) {
  __shared__ long long part[1024];
  const int T = blockDim.x, chunk = (nbox + T - 1) / T;
  const int b = chunk * threadIdx.x, e = min(nbox, b + chunk);
  long long s = 0;
  for (int k = b; k < e; ++k) {
    PairInfo P;
    P.i = P.j = 0;
    for (int a = 0; a < 3; ++a) {
      P.lo[a] = 0;
      P.k[a] = 0;
      P.ext[a] = ext[3 * k + a];
    }
    P.n = P.ext[0] * P.ext[1] * P.ext[2];
    boxes[k] = P;
    s += P.n;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < T; ++t) {
      const long long v = part[t];
      part[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  long long pos = part[threadIdx.x];
  for (int k = b; k < e; ++k) {
    voff[k] = pos;
    pos += boxes[k].n;
  }
}

// Longest boxes first: rank by (size desc, index asc).  This is the order
// the std::stable_sort of sea_poisson_batch (api.cu) produces; the two must
// stay identical, since the persistent CG takes boxes in this order and the
// solutions and iteration counts of the two entry points are compared bit
// for bit.
__global__ void k_noalloc_order(const PairInfo* __restrict__ boxes, int nbox,
                                int* __restrict__ order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nbox) return;
  const int mine = boxes[p].n;
  int rank = 0;
  for (int q = 0; q < nbox; ++q) {
    const int o = boxes[q].n;
    rank += (o > mine) || (o == mine && q < p);
  }
  order[rank] = p;
}

// Device address of the scratch on the current device (looked up once).
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= SEA_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" sea_status sea_poisson_batch_noalloc(const double h[3], int n_box, const int* ext,
                                                const double* rhs, double* x, double tol,
                                                int tol_mode, int max_iter, int* iters,
                                                void* cuda_stream) {
  if (!h || n_box < 0 || (n_box > 0 && (!ext || !rhs || !x))) return SEA_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!(h[a] > 0.0)) return SEA_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 1 || (tol_mode != 0 && tol_mode != 1)) return SEA_ERR_ARG;
  if (n_box > SEA_NOALLOC_MAX_BOXES) return SEA_ERR_LIMIT;
  long long total = 0;
  for (int b = 0; b < n_box; ++b) {
    long long nb = 1;
    for (int a = 0; a < 3; ++a) {
      const int e = ext[3 * b + a];
      if (e < 1 || e > 1024) return SEA_ERR_ARG;
      nb *= e;
    }
    total += nb;
  }
  if (total > SEA_NOALLOC_MAX_UNKNOWNS) return SEA_ERR_LIMIT;
  if (n_box == 0) return SEA_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // a stream under capture cannot take the synchronous copies and the wait
  // below: refuse before anything is queued on it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SEA_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return SEA_ERR_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return SEA_ERR_CUDA;
  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return SEA_ERR_CUDA;
  double* r = (double*)(base + kOffR);
  double* p = (double*)(base + kOffP);
  double* q = (double*)(base + kOffQ);
  PairInfo* boxes = (PairInfo*)(base + kOffBox);
  long long* voff = (long long*)(base + kOffVoff);
  int* order = (int*)(base + kOffOrder);
  int* dit = (int*)(base + kOffIters);
  int* dext = (int*)(base + kOffExt);
  unsigned* status = (unsigned*)(base + kOffMisc);
  int* queue = (int*)(base + kOffMisc + 16);

  cudaError_t e = cudaMemcpyAsync(dext, ext, (size_t)n_box * 3 * sizeof(int),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_noalloc_records<<<1, 1024, 0, st>>>(dext, n_box, boxes, voff);
    k_noalloc_order<<<(n_box + 255) / 256, 256, 0, st>>>(boxes, n_box, order);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = sea::launch_cg_boxes(st, device, h, n_box, boxes, voff, order, rhs, x, r, p, q, dit,
                             status, queue, tol, tol_mode, max_iter);
  unsigned hst = 0;
  if (e == cudaSuccess && iters)
    e = cudaMemcpyAsync(iters, dit, (size_t)n_box * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return SEA_ERR_CUDA;
  return (hst & SEA_FLAG_CG_CAP) ? SEA_ERR_CG_NOT_CONVERGED : SEA_OK;
}
