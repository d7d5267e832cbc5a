// Allocation-free batched inversion of dense complex128 blocks.
//
// Some callers cannot allocate device memory once they are running: an application whose memory
// pool has already reserved the free device memory (a cudaMalloc would fail, or force the pool to
// give back cached blocks), or a latency-bound loop that cannot afford the implicit synchronisation
// of cudaMalloc/cudaFree. This entry point runs the same Gauss-Jordan kernels as hsc_solve's cluster
// inversion, but keeps all of its scratch (pivots, panel copies, GEMM problem lists, error flag) in a
// fixed file-scope device array instead of a workspace allocated per handle. It calls no cudaMalloc,
// cudaFree or other allocating routine.
//
// The array is shared by every call in the process on a given device and keeps the previous call's
// contents; the error flag is cleared at the start of each call, everything else is written before
// it is read. Calls whose work overlaps on the GPU (different streams, or different host threads)
// race on the array and must be serialised by the caller.
//
// The library's translation units are separate CUDA modules, and under lazy module loading (the
// CUDA 12+ default) the array comes into existence when this module is first used on a device, not
// when the library is loaded. The first call on each device therefore loads the module and looks up
// the array's address; a call with batch = 0 does only that, so a caller can make it before its
// memory pool reserves the free device memory and before any stream capture.
#include <atomic>
#include <cstring>

#include "ctx.h"
#include "kernels.cuh"

namespace hsc {
namespace {

constexpr int NA_NB = 16;                // panel width
constexpr int NA_MAX_N = 1024;           // largest block order
constexpr int NA_MAX_ROWS = 8192;        // batch * n
constexpr int NA_MAX_BATCH = 256;
constexpr size_t NA_FLAG_BYTES = 256;
constexpr size_t NA_GJ_BYTES = ((NA_MAX_BATCH * sizeof(GJProb) + 255) / 256) * 256;
constexpr size_t NA_GP_BYTES = ((NA_MAX_BATCH * sizeof(GemmProb) + 255) / 256) * 256;
constexpr size_t NA_PIV_BYTES = ((NA_MAX_ROWS * sizeof(int32_t) + 255) / 256) * 256;
constexpr size_t NA_MR_BYTES = (size_t)NA_MAX_ROWS * 2 * NA_NB * sizeof(c64);
constexpr size_t NA_BYTES = NA_FLAG_BYTES + NA_GJ_BYTES + NA_GP_BYTES + NA_PIV_BYTES + NA_MR_BYTES;

// 4.3 MiB of device scratch, resident on a device from the first call there until process exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the array per device, looked up once (host threads may race on the lookup; they
// store the same value). The cache does not survive cudaDeviceReset: after a reset the address is
// stale, so a process that resets a device must not call this entry point on it again.
constexpr int NA_MAX_DEVICES = 64;
static std::atomic<unsigned char*> g_scratch_ptr[NA_MAX_DEVICES];

__global__ void k_na_setup(GJProb* gj, int n, int batch) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  GJProb p{};
  p.n = n;
  p.ld = n;
  p.off = (int64_t)b * n * n;
  p.piv_off = (int64_t)b * n;
  p.mt_off = (int64_t)b * 2 * n * NA_NB;
  p.rt_off = p.mt_off + (int64_t)n * NA_NB;
  gj[b] = p;
}

// problem list of one trailing-update GEMM step: A^{-1} rows <- M (n x w) R (w x n) + rows outside
// the pivot block
__global__ void k_na_step(GemmProb* gp, int n, int batch, int k0, int w) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  GemmProb p{};
  p.M = n; p.N = n; p.K = w;
  p.a = (int64_t)b * 2 * n * NA_NB; p.lda = NA_NB;
  p.b = p.a + (int64_t)n * NA_NB; p.ldb = n;
  p.c = (int64_t)b * n * n; p.ldc = n;
  p.d = p.c; p.ldd = n;
  p.zr0 = k0; p.zr1 = k0 + w; p.use_d = 1;
  p.tiles_n = (n + 63) / 64;
  p.tile_start = b * ((n + 63) / 64) * p.tiles_n;
  gp[b] = p;
}

}  // namespace
}  // namespace hsc

using namespace hsc;

extern "C" int hsc_block_inverse_noalloc(int32_t n, int32_t batch, const hsc_c128* A,
                                         hsc_c128* Ainv, void* cuda_stream) {
  if (n <= 0 || batch < 0 || (batch > 0 && (!A || !Ainv)))
    return hsc_fail(nullptr, HSC_ERR_ARG, "bad arguments");
  if (n > NA_MAX_N || batch > NA_MAX_BATCH || (int64_t)n * batch > NA_MAX_ROWS)
    return hsc_fail(nullptr, HSC_ERR_ARG,
                    "block inverse without allocation supports n <= 1024, batch <= 256 and "
                    "n * batch <= 8192");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return hsc_fail(nullptr, HSC_ERR_CUDA, "no usable current device");
  unsigned char* base = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!base) {   // once per device, with that device current: loads this module, finds the array
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return hsc_fail(nullptr, HSC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    base = static_cast<unsigned char*>(p);
    g_scratch_ptr[dev].store(base, std::memory_order_release);
  }
  if (batch == 0) return HSC_OK;   // set-up only
  int* flag = reinterpret_cast<int*>(base);
  GJProb* gj = reinterpret_cast<GJProb*>(base + NA_FLAG_BYTES);
  GemmProb* gp = reinterpret_cast<GemmProb*>(base + NA_FLAG_BYTES + NA_GJ_BYTES);
  int32_t* piv = reinterpret_cast<int32_t*>(base + NA_FLAG_BYTES + NA_GJ_BYTES + NA_GP_BYTES);
  c64* MR = reinterpret_cast<c64*>(base + NA_FLAG_BYTES + NA_GJ_BYTES + NA_GP_BYTES + NA_PIV_BYTES);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  c64* out = reinterpret_cast<c64*>(Ainv);
  const size_t bytes = (size_t)batch * n * n * sizeof(c64);
#define NA_CK(call)                                                                              \
  do {                                                                                           \
    cudaError_t _e = (call);                                                                     \
    if (_e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, std::string(#call) + ": " +    \
                                                                  cudaGetErrorString(_e));       \
  } while (0)
  NA_CK(cudaMemsetAsync(flag, 0, NA_FLAG_BYTES, s));
  if ((const void*)A != (const void*)Ainv)
    NA_CK(cudaMemcpyAsync(out, A, bytes, cudaMemcpyDeviceToDevice, s));
  k_na_setup<<<(batch + 127) / 128, 128, 0, s>>>(gj, n, batch);
  NA_CK(cudaGetLastError());
  const int tiles = batch * ((n + 63) / 64) * ((n + 63) / 64);
  for (int k0 = 0; k0 < n; k0 += NA_NB) {
    const int w = n - k0 < NA_NB ? n - k0 : NA_NB;
    NA_CK(launch_gj_panel(gj, batch, out, 0, piv, 0, MR, MR, 0, k0, NA_NB, 1, flag, s));
    NA_CK(launch_gj_swap(gj, batch, n, out, 0, piv, 0, MR, 0, k0, NA_NB, 1, s));
    k_na_step<<<(batch + 127) / 128, 128, 0, s>>>(gp, n, batch, k0, w);
    NA_CK(cudaGetLastError());
    GemmArgs g{};
    g.probs = gp; g.nprob = batch; g.total_tiles = tiles;
    g.A = MR; g.a_es = 0; g.B = MR; g.b_es = 0; g.C = out; g.c_es = 0; g.D = out; g.d_es = 0;
    g.ar = 1.0; g.ai = 0.0; g.br = 1.0; g.bi = 0.0; g.opa = OP_N; g.opb = OP_N;
    NA_CK(gemm_z(g, 1, s));
  }
  NA_CK(launch_gj_colperm(gj, batch, n, out, 0, piv, 0, 1, s));
  int hflag = 0;
  NA_CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  if (hflag) return hsc_fail(nullptr, HSC_ERR_SINGULAR, "zero pivot in a block");
  return HSC_OK;
}
