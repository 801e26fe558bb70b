// noalloc.cu -- mtp_elite_update_noalloc: the elite selection and update of
// mtp_elite_update for callers that must not allocate device memory (for
// example code running inside a memory pool it does not own, or a process
// whose allocator is locked down), so they cannot create a handle.  The
// caller passes every input and output; the intermediate results (weights,
// elite indices, u*, the FP32 copies of the new mean and spread) live in one
// file-scope device array.
#include <mutex>
#include <string>

#include "mtp_device.cuh"

namespace {

// layout of the shared scratch, in bytes
constexpr size_t kWeightOff = 0;
constexpr size_t kEliteOff = kWeightOff + sizeof(double) * MTP_NOALLOC_MAX_ELITES;
constexpr size_t kUstarOff = kEliteOff + sizeof(int32_t) * MTP_NOALLOC_MAX_ELITES;
constexpr size_t kMuOff = kUstarOff + 256;
constexpr size_t kSigmaOff = kMuOff + sizeof(float) * MTP_NOALLOC_MAX_HN;
constexpr size_t kScratchBytes = kSigmaOff + sizeof(float) * MTP_NOALLOC_MAX_HN;

// Resident on every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

mtp_status reject(mtp_status st, const std::string& msg) {
  mtp::set_thread_error(msg);  // readable through mtp_last_error(NULL)
  return st;
}

// Device address of g_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
mtp_status scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return reject(MTP_ERR_CUDA, "elite_update_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      return reject(MTP_ERR_CUDA, std::string("elite_update_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
    e = mtp::init_select_attributes();
    if (e != cudaSuccess)
      return reject(MTP_ERR_CUDA, std::string("elite_update_noalloc: kernel attributes: ") +
                                      cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MTP_OK;
}

}  // namespace

extern "C" mtp_status mtp_elite_update_noalloc(const float* d_cost, const float* d_U, int32_t B,
                                               int32_t E, int32_t H, int32_t n, double lambda,
                                               double alpha, double sigma_min, int32_t update_rule,
                                               double* d_mu, double* d_sigma, int32_t* d_elite,
                                               float* d_ustar, void* stream) {
  if (!d_cost || !d_U || !d_mu || !d_sigma)
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: null input pointer");
  if (B < 1 || E < 1 || E > B || H < 1 || n < 1 || n > MTP_MAX_CTRL)
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: need 1 <= E <= B, H >= 1, 1 <= n <= 32");
  if (E > MTP_NOALLOC_MAX_ELITES)
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: E exceeds MTP_NOALLOC_MAX_ELITES");
  if ((long long)H * n > MTP_NOALLOC_MAX_HN)
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: H*n exceeds MTP_NOALLOC_MAX_HN");
  if (mtp::select_smem_bytes(B, E) > 200 * 1024)
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: B too large for the one-block selection");
  if (!(lambda > 0.0) || !(alpha >= 0.0 && alpha < 1.0) || !(sigma_min > 0.0) ||
      (update_rule != MTP_UPDATE_SOFTMAX && update_rule != MTP_UPDATE_PLAIN_CEM))
    return reject(MTP_ERR_INVALID_ARG, "elite_update_noalloc: bad lambda / alpha / sigma_min / rule");
  unsigned char* base = nullptr;
  mtp_status st = scratch_on_current_device(&base);
  if (st != MTP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* weight = reinterpret_cast<double*>(base + kWeightOff);
  int32_t* elite = reinterpret_cast<int32_t*>(base + kEliteOff);
  float* ustar = reinterpret_cast<float*>(base + kUstarOff);
  float* mu_f = reinterpret_cast<float*>(base + kMuOff);
  float* sigma_f = reinterpret_cast<float*>(base + kSigmaOff);
  mtp::SelectArgs sa{d_cost, d_U, B, E, H, n, 1.0 / lambda, update_rule,
                     elite, weight, ustar, d_elite, d_ustar};
  cudaError_t e = mtp::launch_select(sa, s);
  if (e != cudaSuccess)
    return reject(MTP_ERR_CUDA, std::string("elite_update_noalloc: select: ") + cudaGetErrorString(e));
  mtp::UpdateArgs ua{d_U, elite, weight, E, H, n, alpha, sigma_min, update_rule,
                     d_mu, d_sigma, mu_f, sigma_f, nullptr};
  e = mtp::launch_update(ua, s);
  if (e != cudaSuccess)
    return reject(MTP_ERR_CUDA, std::string("elite_update_noalloc: update: ") + cudaGetErrorString(e));
  return MTP_OK;
}
