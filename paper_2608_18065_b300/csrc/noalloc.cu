// noalloc.cu -- nqs_logpsi_noalloc: log Psi of given configurations with
// no device allocation at all, for callers that cannot call cudaMalloc.
//
// Who needs this: code that must not allocate device memory at the point it
// evaluates the wave function -- for example a host framework whose memory
// pool already owns the whole device, a plug-in that may only use memory it
// was handed, or a real-time loop where an allocation (and the implicit
// device synchronisation it can cause) is not allowed.  Such a caller cannot
// create the torch/cudaMalloc workspace that nqs_logpsi expects.
//
// How: the two scratch buffers that the log Psi kernels need beyond their
// inputs and outputs -- the packed copy of theta and the per-site hidden-
// state cache (read back for the vertical neighbours of 2D lattices) --
// live in one file-scope __device__ array of NQS_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads the library reserves that array until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and passes it to the kernels.
#include <mutex>

#include "launch.h"
#include "pack.cuh"

using namespace nqs;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NQS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once
// per device).
nqs_status scratch_for_current_device(void **ptr, int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NQS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NQS_ERR_CUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return NQS_ERR_CUDA;
    g_scratch_addr[dev] = p;
    g_sm_count[dev] = n;
  }
  *ptr = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return NQS_OK;
}

}  // namespace

extern "C" nqs_status nqs_logpsi_noalloc(const nqs_model_desc *model, const double *theta,
                                         const uint8_t *spins, int64_t n, double *logpsi,
                                         void *stream) {
  if (!model || !theta || !spins || !logpsi || n <= 0) return NQS_ERR_ARG;
  const nqs_model_desc &m = *model;
  if (m.dim != 1 && m.dim != 2) return NQS_ERR_ARG;
  if (m.Lx <= 0 || m.Ly <= 0 || (m.dim == 1 && m.Ly != 1)) return NQS_ERR_ARG;
  const int64_t N = (int64_t)m.Lx * m.Ly;
  if (N < 2 || N > 4096 || (m.zmask && (N % 2))) return NQS_ERR_ARG;
  if (!dh_supported(m.dh)) return NQS_ERR_UNSUPPORTED;
  const Layout L = make_layout(m);
  const PackOff P = pack_offsets(L);
  // scratch: packed theta (FP64), then, for 2D lattices only, the hidden-
  // state cache [n][N][dh] (FP64) that the vertical neighbours read back; a
  // 1D chain reads no earlier state, so it needs the packed weights alone
  const size_t cap = (size_t)NQS_NOALLOC_SCRATCH_BYTES;
  const size_t pack_bytes = al256((size_t)P.total * sizeof(double));
  if (pack_bytes > cap) return NQS_ERR_WORKSPACE;
  const size_t row_bytes = (size_t)N * m.dh * sizeof(double);
  const bool need_cache = m.dim == 2;
  // n is compared before it is multiplied, so the product cannot wrap
  if (need_cache && (size_t)n > (cap - pack_bytes) / row_bytes) return NQS_ERR_WORKSPACE;
  if ((size_t)n > (size_t)INT32_MAX) return NQS_ERR_WORKSPACE;
  void *scratch = nullptr;
  int sms = 0;
  nqs_status s = scratch_for_current_device(&scratch, &sms);
  if (s != NQS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *pack = static_cast<double *>(scratch);
  double *hcache = need_cache
      ? reinterpret_cast<double *>(static_cast<unsigned char *>(scratch) + pack_bytes)
      : nullptr;
  // Every scratch element a kernel reads is written earlier in the same call
  // (the pack first, each cached state before its vertical neighbour reads
  // it), so nothing has to be cleared between calls.
  const int blocks = (int)min64((P.total + 255) / 256, 4096);
  k_pack<double><<<blocks, 256, 0, st>>>(theta, pack, L, P);
  if (cudaGetLastError() != cudaSuccess) return NQS_ERR_CUDA;
  FwdArgs<double> a{};
  a.pack = pack;
  a.N = (int)N; a.Lx = m.Lx; a.cplx = m.cplx; a.marshall = m.marshall; a.zmask = m.zmask;
  a.nrows = n;
  a.spins = const_cast<uint8_t *>(spins);
  a.logpsi = logpsi;
  a.hcache = hcache;
  a.lccache = nullptr;
  const RecDesc d{m.dim, m.dh, (int)N, m.Lx, m.cplx, m.marshall, m.zmask, sms};
  return run_forward<double>(d, MODE_GIVEN, a, 0, st) == cudaSuccess ? NQS_OK : NQS_ERR_CUDA;
}
