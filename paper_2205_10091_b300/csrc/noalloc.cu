// Allocation-free Pauli-sum energies: tc_expect_pauli_sum_noalloc.
//
// Some callers cannot allocate device memory at the point where they need an
// energy: code that runs under a fixed memory reservation, inside an
// allocator callback, or in a real-time loop where cudaMalloc's implicit
// synchronisation is not acceptable.  This entry point computes the same
// energies as tc_expect_pauli_sum but keeps its scratch (the compiled Pauli-sum
// plan and the per-tile partial sums) in one file-scope __device__ array of a
// fixed size, so it never calls cudaMalloc, cudaFree or any allocating routine.
#include <cstring>
#include <mutex>
#include <string>

#include "engine.h"

namespace {

// 8 MiB of scratch.  Every GPU that loads this library holds it until exit.
constexpr size_t kScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array for the current device.  In host code
// `g_noalloc_scratch` is only a host-side stand-in for the symbol, never a
// device address; the real address comes from cudaGetSymbolAddress, taken
// once per device with that device current (on the first call there).  The
// cached address belongs to the device's primary context: the library must
// not be used on a device after cudaDeviceReset there.
tc_status scratch_for_device(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return tcb::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TC_OK;
}
}  // namespace

using namespace tcb;

extern "C" tc_status tc_expect_pauli_sum_noalloc(const tc_circuit* c, const void* d_states, int B,
                                                 const uint8_t* structures, const double* weights, int T,
                                                 double* d_energy_out, void* stream) {
  if (!c || (B != 0 && (!d_states || !d_energy_out))) return fail(TC_E_INVALID, "NULL argument");
  if (B < 0 || T < 0) return fail(TC_E_INVALID, "B < 0 or T < 0");
  if (T > 0 && (!structures || !weights)) return fail(TC_E_INVALID, "structures/weights are NULL");
  if (c->N != c->n) return fail(TC_E_UNSUPPORTED, "the allocation-free entry point needs n >= 10");

  // Set-up comes before the B == 0 return, so that a call with no rows can
  // serve as the warm-up: the first lookup on a device loads this file's
  // module, and with it the scratch array, which may allocate device memory.
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(TC_E_UNSUPPORTED, "device index beyond 63");
  void* base = nullptr;
  tc_status st = scratch_for_device(dev, &base);
  if (st != TC_OK) return st;
  if (B == 0) return TC_OK;
  // the plan is copied from host memory that is freed when the call returns:
  // a captured copy node would read it later, so capture is refused
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing((cudaStream_t)stream, &cs)) != cudaSuccess) return cuda_fail(e, "capture query");
    if (cs != cudaStreamCaptureStatusNone)
      return fail(TC_E_UNSUPPORTED, "the allocation-free entry point cannot be captured into a graph");
  }

  // compile the Pauli sum on the host (host memory only)
  HamPlan H;
  std::string err;
  if (!build_hamiltonian(c->n, c->N, c->k_ham, structures, weights, T, H, err))
    return fail(err.find("flips more") != std::string::npos ? TC_E_UNSUPPORTED : TC_E_INVALID, err);
  const int nh = (int)H.passes.size();
  const size_t tiles_h = (size_t)1 << (c->N - c->k_ham);
  const size_t o_pass = 0;
  const size_t o_hdiag = o_pass + align256(H.passes.size() * sizeof(DevPass));
  const size_t o_hterm = o_hdiag + align256(H.hdiag.size() * sizeof(DevHDiag));
  const size_t o_hflip = o_hterm + align256(H.hterms.size() * sizeof(DevHTerm));
  const size_t o_epart = o_hflip + align256(H.hflips.size() * sizeof(DevHFlip));
  const size_t need = o_epart + (size_t)B * nh * tiles_h * sizeof(double);
  if (need > kScratchBytes)
    return fail(TC_E_INVALID, "allocation-free Pauli sum needs " + std::to_string(need) +
                                  " bytes of scratch; the fixed limit is " + std::to_string(kScratchBytes) +
                                  " (use fewer rows per call)");

  char* sc = (char*)base;
  cudaStream_t s = (cudaStream_t)stream;

  // the plan is rewritten on every call; partial sums are fully overwritten
  auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(sc + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  if ((e = put(o_pass, H.passes.data(), H.passes.size() * sizeof(DevPass))) != cudaSuccess ||
      (e = put(o_hdiag, H.hdiag.data(), H.hdiag.size() * sizeof(DevHDiag))) != cudaSuccess ||
      (e = put(o_hterm, H.hterms.data(), H.hterms.size() * sizeof(DevHTerm))) != cudaSuccess ||
      (e = put(o_hflip, H.hflips.data(), H.hflips.size() * sizeof(DevHFlip))) != cudaSuccess)
    return cuda_fail(e, "plan copy to scratch");

  KArgs a{};
  a.hpasses = (const DevPass*)(sc + o_pass);
  a.hdiag = (const DevHDiag*)(sc + o_hdiag);
  a.hterms = (const DevHTerm*)(sc + o_hterm);
  a.hflips = (const DevHFlip*)(sc + o_hflip);
  a.N = c->N;
  a.n_user = c->n;
  a.psi = const_cast<void*>(d_states);
  a.lam = nullptr;
  a.store_lambda = 0;
  a.epart = (double*)(sc + o_epart);
  a.n_hpasses = nh;
  const bool dbl = c->dtype == TC_C128;
  for (int p = 0; p < nh; ++p) {
    a.pass = p;
    if ((e = launch_pass(KM_HAM, dbl, a, H.passes[p], nullptr, B, s)) != cudaSuccess) return cuda_fail(e, "pauli-sum pass");
  }
  if ((e = launch_finalize(a.epart, nh, (int)tiles_h, nullptr, 0, 1, nullptr, nullptr, 0, B, d_energy_out, nullptr,
                           s)) != cudaSuccess)
    return cuda_fail(e, "finalize");
  return TC_OK;
}
