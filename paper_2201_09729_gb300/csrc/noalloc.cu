// dlma_apply_schur_noalloc: the even-odd Schur operator for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte
// of device memory through its own pool and forbids allocations it does not
// account for, or a caller that cannot accept the device-wide synchronisation
// cudaMalloc / cudaFree may imply in the middle of its own work.  For them
// this entry point allocates nothing.  Its work space -- the packed input, the
// odd-site intermediate T_oo^-1 D_oe in and the packed output -- lives in one
// file-scope __device__ array of a fixed size, held until the process exits by
// every GPU that has loaded the library's device code.  That code is loaded
// lazily, per device, so the array is reserved on a device by the first call
// there (the same call that looks up its address, below).
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so its device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, and passed to the
// kernels.  That set-up happens in the first call on each device; make that
// first call before any stream capture.  Nothing in the work space has to
// start at zero: every call overwrites all of the packed input, the
// intermediate and the packed output before reading them.  All calls share the
// one array, which keeps the last call's contents; calls that overlap on the
// GPU (two streams, two contexts on one device, two host threads) race on it.
#include "common.cuh"
#include <mutex>

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_schur_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

dlma_status scratch_address(dlma_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "device index %d out of range for the static work space", ctx->device);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[ctx->device]) {
    CU(cudaSetDevice(ctx->device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_schur_scratch);
    if (e != cudaSuccess || !p)
      return set_err(ctx, DLMA_ERR_CUDA, "cudaGetSymbolAddress of the static work space failed: %s",
                     cudaGetErrorString(e));
    g_addr[ctx->device] = p;
  }
  *out = g_addr[ctx->device];
  return DLMA_OK;
}

}  // namespace

extern "C" dlma_status dlma_apply_schur_noalloc(dlma_ctx* ctx, const double* in, double* out, int nrhs, int dagger) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params)
    return set_err(ctx, DLMA_ERR_STATE, "gauge field and parameters must be set first");
  if (!in || !out || nrhs < 1) return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_apply_schur_noalloc");
  const size_t field = field_bytes_per_rhs(DLMA_FP64, ctx->g.Vh) * (size_t)nrhs;
  const size_t need = 3 * field;
  if (need > kScratchBytes)
    return set_err(ctx, DLMA_ERR_INVALID_ARG,
                   "dlma_apply_schur_noalloc: %d right-hand sides of %d even sites need %zu bytes of work space, "
                   "above the fixed %zu bytes; use at most %zu right-hand sides or dlma_apply_schur",
                   nrhs, ctx->g.Vh, need, kScratchBytes, kScratchBytes / (3 * field_bytes_per_rhs(DLMA_FP64, ctx->g.Vh)));
  void* base = nullptr;
  TRY(scratch_address(ctx, &base));
  CU(cudaSetDevice(ctx->device));
  Field fin, tmp, fout;
  fin.prec = tmp.prec = fout.prec = DLMA_FP64;
  fin.nrhs = tmp.nrhs = fout.nrhs = nrhs;
  fin.Vh = tmp.Vh = fout.Vh = ctx->g.Vh;
  fin.data = base;
  tmp.data = (char*)base + field;
  fout.data = (char*)base + 2 * field;
  TRY(pack_parity(ctx, in, 0, 0, fin));
  TRY(schur_apply(ctx, fin, tmp, fout, dagger ? 1 : 0, nullptr, nullptr));
  TRY(unpack_parity(ctx, fout, 0, 0, out));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}
