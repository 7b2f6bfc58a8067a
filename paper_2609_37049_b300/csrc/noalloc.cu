// lqcd_disc_correlator_noalloc: the disconnected-correlator computation of
// lqcd_disc_correlator for callers that must not allocate GPU memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not safe -- a host
// application that reserves all device memory up front and forbids later allocations (a memory
// pool owner, a framework that hands out fixed arenas), or a latency-critical loop where an
// allocation would synchronise the device.  Such a caller owns
// every input and output buffer; the only extra memory this computation needs -- the
// differences dL = L - L_Lambda and dLt = Lt - Lt_Lambda for the four-piece split -- lives in
// the fixed array below, which the CUDA runtime places in device memory when the library is
// loaded and which stays allocated on every GPU that loads the library until the process exits.
#include <mutex>
#include <string>

#include "lqcd_distill.h"

namespace lqcd {
void set_global_error(const std::string& msg);
}

using namespace lqcd;

// Largest n_cfg * n_gamma * Lt the scratch holds (two complex arrays of this many entries, 2 MiB).
#define LQCD_NOALLOC_MAX_LOOP_ENTRIES (1 << 16)

static __device__ __align__(256) double2 g_noalloc_scratch[2 * LQCD_NOALLOC_MAX_LOOP_ENTRIES];

namespace {
// Device address of the scratch array per device: in host code the symbol name only stands for
// the array, it is not a device address, so it is looked up once per device with that device
// current and the looked-up pointer is what the kernels get.
constexpr int kMaxDevices = 64;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_global_error("disc_correlator_noalloc: no usable current CUDA device");
    return LQCD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_global_error(std::string("disc_correlator_noalloc: cudaGetSymbolAddress failed: ") +
                       cudaGetErrorString(e));
      return LQCD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LQCD_OK;
}
}  // namespace

extern "C" int lqcd_disc_correlator_noalloc(const double* L, const double* Lt, const double* Ld, const double* Ltd,
                                            int n_cfg, int n_gamma, int T, const int* dom_of_t, int vev, double* C,
                                            double* Cdd, double* dC, double* C_avg, double* dC_avg, int* valid,
                                            int* n_valid, double* terms, void* stream) {
  if (!L || !Lt || !Ld || !Ltd || !dom_of_t || !C || !Cdd || !dC || !C_avg || !dC_avg || !valid || !n_valid ||
      n_cfg < 1 || n_gamma < 1 || T < 1) {
    set_global_error("disc_correlator_noalloc: bad arguments");
    return LQCD_ERR_INVALID_ARG;
  }
  if (T > LQCD_MAXT) {
    set_global_error("disc_correlator_noalloc: Lt > 256");
    return LQCD_ERR_INVALID_ARG;
  }
  if (vev && n_cfg < 2) {
    set_global_error("disc_correlator_noalloc: the VEV subtraction needs n_cfg >= 2");
    return LQCD_ERR_INVALID_ARG;
  }
  const long entries = (long)n_cfg * n_gamma * T;
  if (terms && entries > LQCD_NOALLOC_MAX_LOOP_ENTRIES) {
    set_global_error("disc_correlator_noalloc: n_cfg * n_gamma * Lt = " + std::to_string(entries) +
                     " exceeds the fixed scratch of 65536 entries; use lqcd_disc_correlator");
    return LQCD_ERR_INVALID_ARG;
  }
  double2* scratch = nullptr;
  if (int rc = scratch_for_current_device(&scratch)) return rc;
  // dL and dLt are written in full by this call before they are read, so nothing has to be
  // cleared between calls.
  double2* dL = scratch;
  double2* dLt = scratch + LQCD_NOALLOC_MAX_LOOP_ENTRIES;
  cudaStream_t st = (cudaStream_t)stream;
  correlators((const double2*)L, (const double2*)Lt, (const double2*)Ld, (const double2*)Ltd, n_cfg, n_gamma, T, vev,
              dom_of_t, (double2*)C, (double2*)Cdd, (double2*)dC, (double2*)C_avg, (double2*)dC_avg, valid, n_valid,
              (double2*)terms, dL, dLt, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("disc_correlator_noalloc: ") + cudaGetErrorString(e));
    return LQCD_ERR_CUDA;
  }
  return LQCD_OK;
}
