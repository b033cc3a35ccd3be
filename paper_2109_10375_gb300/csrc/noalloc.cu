// amber_rank_noalloc: the ranking of amber_rank for callers that cannot
// allocate device memory, with its working storage in a fixed array that the
// library itself carries.
//
// Who needs it: code that runs where cudaMalloc is off limits or unsafe -- a
// plug-in living inside another framework that owns the whole device pool, a
// hard real-time loop that must never hit an allocation (cudaMalloc can
// synchronise the device), or a process started with its memory budget already
// handed out.  Such callers own their inputs and outputs but have nowhere to
// put the sort's ping-pong buffers and look-back state.
//
// The scratch is one file-scope __device__ array of fixed size, so every GPU
// that loads the library holds it (about 17 MB) until the process exits, and
// ranks of at most kNoAllocMaxCells cells fit.  Host code cannot use the
// array's name as a device address (it names a host-side stand-in), so the
// first call on each device looks the address up with cudaGetSymbolAddress
// while that device is current and caches it.
#include <mutex>

#include "sort.cuh"

namespace amber {
namespace {

constexpr int64_t kNoAllocMaxCells = (int64_t)1 << 20;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// layout of the scratch array
constexpr size_t kKeyBytes = align_up((size_t)kNoAllocMaxCells * 4);
constexpr size_t kLookbackWords = (size_t)((kNoAllocMaxCells + kTile - 1) / kTile) * kMaxRadix;
constexpr size_t kOffKeysA = 0;
constexpr size_t kOffKeysB = kOffKeysA + kKeyBytes;
constexpr size_t kOffIdxA = kOffKeysB + kKeyBytes;
constexpr size_t kOffIdxB = kOffIdxA + kKeyBytes;
constexpr size_t kOffLookback = kOffIdxB + kKeyBytes;
constexpr size_t kOffCtrl = kOffLookback + align_up(2 * kLookbackWords * 4);
constexpr size_t kOffStatus = kOffCtrl + align_up(sizeof(SortCtrl));
constexpr size_t kScratchBytes = kOffStatus + kAlign;

static __device__ __align__(256) unsigned char g_rank_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

}  // namespace
}  // namespace amber

using namespace amber;

extern "C" int amber_rank_noalloc(const float* d_J, int64_t ncells, uint32_t* d_order, unsigned int* d_status_opt,
                                  void* stream) {
  // arrays start on their element size (checked before any CUDA call)
  if (!d_J || !d_order || ncells < 1 || (reinterpret_cast<uintptr_t>(d_J) & 3) != 0 ||
      (reinterpret_cast<uintptr_t>(d_order) & 3) != 0 || (reinterpret_cast<uintptr_t>(d_status_opt) & 3) != 0)
    return AMBER_ERR_INVALID_ARG;
  if (ncells > kNoAllocMaxCells) return AMBER_ERR_CAPACITY;  // the fixed scratch holds 2^20 cells
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  unsigned char* base;
  int sms;
  {
    // once per device, with that device current: resolve the array's device address
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_rank_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return AMBER_ERR_CUDA;
      }
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return AMBER_ERR_CUDA;
      }
      g_num_sms[dev] = n;
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    sms = g_num_sms[dev];
  }
  SortWork w{};
  w.keysA = base + kOffKeysA;
  w.keysB = base + kOffKeysB;
  w.idxA = reinterpret_cast<uint32_t*>(base + kOffIdxA);
  w.idxB = reinterpret_cast<uint32_t*>(base + kOffIdxB);
  w.massA = w.massB = nullptr;
  w.lookback = reinterpret_cast<uint32_t*>(base + kOffLookback);
  w.ctrl = reinterpret_cast<SortCtrl*>(base + kOffCtrl);
  w.max_cells = kNoAllocMaxCells;
  w.num_sms = sms;
  unsigned int* status = d_status_opt ? d_status_opt : reinterpret_cast<unsigned int*>(base + kOffStatus);
  // rank_impl clears everything that must start at zero (control block,
  // tickets, look-back regions) with stream-ordered memsets and kernels
  const cudaError_t e = rank_impl<float>(w, d_J, ncells, d_order, nullptr, nullptr, nullptr, false, status,
                                         (cudaStream_t)stream, nullptr, kSpinLimit);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  return AMBER_OK;
}
