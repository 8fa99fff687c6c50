// H psi without any device allocation: pw_hamiltonian_apply_noalloc.
//
// Who needs it: code that may not call cudaMalloc / cudaFree at the point where
// it applies H -- for instance a host framework whose caching allocator already
// owns the device memory and forbids foreign allocations, a caller running under
// a hard device-memory cap, or a latency-critical loop that cannot afford the
// device-wide synchronisation cudaFree implies.  The context itself is built
// beforehand (pw_ctx_create allocates); this entry point then reuses one
// fixed, file-scope device array as its only scratch.
//
// The scratch: `g_noalloc_scratch`, kNoallocScratchBytes (32 MiB), resident on
// every GPU that loads this library until the process exits.  Host code never
// dereferences the symbol; it obtains the device address once per device with
// cudaGetSymbolAddress (done on the first call on that device, so that first call
// must happen before any stream capture) and passes it to the kernels.  The cached
// address belongs to the device's primary context: after cudaDeviceReset it is stale,
// so a process that resets a device must not call this entry point on it again.
// Every call shares the array and leaves its last contents behind; calls that
// overlap on the GPU (different streams, different host threads) race on it.
// No part of it has to start at zero: each kernel writes the region it reads
// later in the same call.
#include <algorithm>
#include <mutex>

#include "pw_internal.cuh"

namespace pw {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (set up once per device)
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(PW_EUNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return PW_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

}  // namespace pw

using namespace pw;

extern "C" PW_API int pw_hamiltonian_apply_noalloc(pw_ctx* ctx, const void* psi_v, int64_t ldpsi, int nband,
                                                   void* hpsi_v, int64_t ldout) {
  if (!ctx) return set_error(PW_EINVAL, "NULL context");
  if (ctx->poisoned) return set_error(PW_ECUDA, "context poisoned by an earlier CUDA error");
  if (nband < 0) return set_error(PW_EINVAL, "nband < 0");
  if (nband == 0) return PW_OK;
  if (!psi_v || !hpsi_v) return set_error(PW_EINVAL, "NULL block");
  if (ldpsi < ctx->npw || ldout < ctx->npw) return set_error(PW_EINVAL, "ld < npw (%d)", ctx->npw);
  if (psi_v == hpsi_v) return set_error(PW_EINVAL, "psi aliases hpsi");
  const double2* psi = (const double2*)psi_v;
  double2* hpsi = (double2*)hpsi_v;
  const int npw = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  // scratch per band: half-box planes + C_proj + Z; per chunk: split-K partials (nsplit x np x nb)
  const int nsplit = 8;
  const size_t hb_band = (size_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2] * sizeof(double2);
  const size_t cz_band = (size_t)np * sizeof(double2);
  const size_t per_band = align256(hb_band) + 2 * align256(cz_band) + align256((size_t)nsplit * cz_band);
  if (per_band > kNoallocScratchBytes)
    return set_error(PW_EINVAL, "one band needs %zu bytes of scratch; the static scratch holds %zu bytes", per_band,
                     kNoallocScratchBytes);
  const int chunk = (int)std::min<size_t>((size_t)nband, kNoallocScratchBytes / per_band);
  void* base = nullptr;
  int s = noalloc_scratch(&base);
  if (s != PW_OK) return s;
  unsigned char* p = (unsigned char*)base;
  double2* hb = (double2*)p;
  p += align256(hb_band * chunk);
  double2* Cm = (double2*)p;
  p += align256(cz_band * chunk);
  double2* Z = (double2*)p;
  p += align256(cz_band * chunk);
  double2* spl = (double2*)p;
  for (int b0 = 0; b0 < nband; b0 += chunk) {
    const int nb = std::min(chunk, nband - b0);
    const double2* x = psi + (int64_t)b0 * ldpsi;
    double2* y = hpsi + (int64_t)b0 * ldout;
    cudaError_t e = launch_local_apply<double>(ctx->plan, ctx->tw64, ctx->sp, ctx->vperm64, ctx->kin64, x, ldpsi, nb,
                                               y, ldout, hb, nb, st, nullptr);
    if (e == cudaSuccess && np > 0) {
      Epi<double> ec;
      ec.mode = EPI_STORE; ec.out = Cm; ec.ldo = np; ec.alpha = 1.0; ec.beta = 0; ec.shift = 0;
      ec.yk = nullptr; ec.ykm1 = nullptr; ec.ldy = 0; ec.ldy2 = 0; ec.dev_ce = nullptr; ec.first = 0;
      e = launch_cgemm<double>(1, 0, np, nb, npw, ctx->P64, npw, x, ldpsi, ec, nsplit, spl, st);
      if (e == cudaSuccess)
        e = launch_dblock<double>(np, nb, ctx->D64, ctx->blk0, ctx->blklen, Cm, np, Z, np, st);
      if (e == cudaSuccess) {
        Epi<double> ea = ec;
        ea.mode = EPI_ACCUM; ea.out = y; ea.ldo = ldout;
        e = launch_cgemm<double>(0, 0, npw, nb, np, ctx->P64, npw, Z, np, ea, 1, nullptr, st);
      }
    }
    if (e != cudaSuccess) {
      ctx->poisoned = true;
      return cuda_status(e, "no-alloc H apply");
    }
  }
  return PW_OK;
}
