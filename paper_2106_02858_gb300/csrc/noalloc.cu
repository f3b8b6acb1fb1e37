// cmcg_inner_noalloc: the (eps, mu)-weighted inner product of two nodal fields
// without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// need the inner product -- code that owns all device memory through its own
// pool allocator (a framework's caching allocator), code running between
// stream-ordered work that must not be serialised (cudaMalloc and cudaFree can
// synchronise the device), and callers without a handle, since cmcg_create
// allocates the whole solver state.  The handle-based cmcg_inner reduces
// through a per-handle block-partials buffer allocated by cmcg_create; this
// variant reduces through one file-scope array instead.
//
// The array (NA_MAX_BLOCKS doubles, 64 KiB) is static device memory: every
// GPU that loads the library holds it until the process exits.  Host code only
// ever sees a stand-in for its name, so the device address is fetched with
// cudaGetSymbolAddress once per device, with that device current, and passed
// to the kernels.  Every call shares the array and finds the previous call's
// contents in it; nothing needs clearing because every entry a call reads was
// written earlier in the same call.  Calls that overlap on the GPU (two streams,
// or two host threads) race on the array.
#include <mutex>

#include "common.h"

namespace cmcg {
namespace {

constexpr int NA_THREADS = 128;        // one tetrahedron per thread, one partial per block
constexpr int NA_MAX_BLOCKS = 8192;    // 8192 doubles = 64 KiB of static scratch
static_assert(int64_t(NA_THREADS) * NA_MAX_BLOCKS == CMCG_NOALLOC_MAX_TETS, "limit mismatch");

static __device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS];

__constant__ double cNaM1[4 * 4];
__constant__ double cNaM2[10 * 10];
__constant__ double cNaM3[20 * 20];

template <int Q>
__device__ __forceinline__ double na_mass(int idx) {
  if constexpr (Q == 1) return cNaM1[idx];
  else if constexpr (Q == 2) return cNaM2[idx];
  else return cNaM3[idx];
}

// Boundary layout: u, v are [tet][6][Np]; w is [tet][2] = (6|K| eps_K, 6|K| mu_K).
template <int Q>
__global__ void __launch_bounds__(NA_THREADS) na_dot_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                                            const double* __restrict__ w, int64_t nt,
                                                            double* __restrict__ partials) {
  constexpr int NP = np_of(Q);
  const int64_t k = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x;
  double acc = 0;
  if (k < nt) {
    const double* uk = u + k * 6 * NP;
    const double* vk = v + k * 6 * NP;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double s = 0;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        double t = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) t = fma(na_mass<Q>(i * NP + j), vk[c * NP + j], t);
        s = fma(uk[c * NP + i], t, s);
      }
      acc += w[2 * k + (c < 3 ? 0 : 1)] * s;
    }
  }
  __shared__ double sh[NA_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < NA_THREADS / 32; ++i) s += sh[i];
    partials[blockIdx.x] = s;
  }
}

__global__ void na_finalize_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

struct NaDevice {
  bool ready = false;
  double* partials = nullptr;  // device address of g_na_partials on this device
};
std::mutex g_na_mutex;
NaDevice g_na_dev[64];

// Once per device, with that device current: upload the reference mass
// matrices and look up the scratch array's device address.
int na_setup(int device, double** partials) {
  std::lock_guard<std::mutex> lk(g_na_mutex);
  NaDevice& d = g_na_dev[device];
  if (!d.ready) {
    const RefMats& r1 = ref_mats(1);
    const RefMats& r2 = ref_mats(2);
    const RefMats& r3 = ref_mats(3);
    if (cudaMemcpyToSymbol(cNaM1, r1.M.data(), sizeof(double) * r1.M.size()) != cudaSuccess ||
        cudaMemcpyToSymbol(cNaM2, r2.M.data(), sizeof(double) * r2.M.size()) != cudaSuccess ||
        cudaMemcpyToSymbol(cNaM3, r3.M.data(), sizeof(double) * r3.M.size()) != cudaSuccess)
      return CMCG_ERR_CUDA;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_partials) != cudaSuccess || p == nullptr) return CMCG_ERR_CUDA;
    d.partials = static_cast<double*>(p);
    d.ready = true;
  }
  *partials = d.partials;
  return CMCG_OK;
}

}  // namespace
}  // namespace cmcg

extern "C" int cmcg_inner_noalloc(int order, int64_t nt, const double* u, const double* v, const double* w,
                                  double* out, void* stream) {
  using namespace cmcg;
  if (order < 1 || order > 3 || nt < 1 || !u || !v || !w || !out) return CMCG_ERR_INVALID_ARG;
  if (nt > CMCG_NOALLOC_MAX_TETS) return CMCG_ERR_INVALID_ARG;  // beyond the static scratch
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return CMCG_ERR_NO_DEVICE;
  if (device < 0 || device >= 64) return CMCG_ERR_INVALID_ARG;
  double* partials = nullptr;
  int rc = na_setup(device, &partials);
  if (rc != CMCG_OK) return rc;
  const int nblocks = int((nt + NA_THREADS - 1) / NA_THREADS);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (order == 1) na_dot_kernel<1><<<nblocks, NA_THREADS, 0, s>>>(u, v, w, nt, partials);
  else if (order == 2) na_dot_kernel<2><<<nblocks, NA_THREADS, 0, s>>>(u, v, w, nt, partials);
  else na_dot_kernel<3><<<nblocks, NA_THREADS, 0, s>>>(u, v, w, nt, partials);
  na_finalize_kernel<<<1, 256, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError() == cudaSuccess ? CMCG_OK : CMCG_ERR_CUDA;
}
