// noalloc.cu -- an allocation-free variant of the CIC deposit.
//
// Some callers cannot allocate device memory on their own: a host application that
// hands the library a fixed memory budget reserved up front (for instance when a
// framework's caching allocator already owns the device memory), or a plug-in
// environment that forbids runtime allocations after start-up.  For them the int64
// fixed-point accumulator of the deposit lives in a file-scope device array of fixed
// size, which every GPU that loads this library holds until the process exits.  The
// caller still provides the positions and the output grid.
#include <mutex>

#include "internal.cuh"

namespace pmeft {

constexpr int kStaticMaxN = 128;  // largest mesh the static accumulator holds
constexpr size_t kStaticCells = (size_t)kStaticMaxN * kStaticMaxN * kStaticMaxN;  // 16 MiB of int64

static __device__ __align__(256) unsigned long long g_static_acc[kStaticCells];
static __device__ __align__(256) int g_static_flag[64];

// Host-side device addresses of the two arrays, one entry per device, filled on the
// first call on that device (the array names are host-side stand-ins in host code).
struct StaticSlot {
    bool ready = false;
    unsigned long long* acc = nullptr;
    int* flag = nullptr;
    int sms = 0;
};
static std::mutex g_static_mu;
static StaticSlot g_static_slots[64];

void launch_deposit_on(cudaStream_t s, int sms, const double* pos, long long np, int n, unsigned long long* acc);
void launch_density_on(cudaStream_t s, int sms, const long long* acc, int n, long long np, double* delta, int* flag);

}  // namespace pmeft

using namespace pmeft;

extern "C" pm_status pm_deposit_cic_static(const double* pos, long long np, int n, double* delta, void* cuda_stream)
{
    if (!pos || !delta || np < 1 || !valid_n(n)) return PM_ERR_INVALID_ARG;
    if (n > kStaticMaxN) return PM_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PM_ERR_CUDA;
    StaticSlot slot;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        StaticSlot& sl = g_static_slots[dev];
        if (!sl.ready) {
            // once per device, with that device current
            void* a = nullptr;
            void* f = nullptr;
            if (cudaGetSymbolAddress(&a, g_static_acc) != cudaSuccess) return PM_ERR_CUDA;
            if (cudaGetSymbolAddress(&f, g_static_flag) != cudaSuccess) return PM_ERR_CUDA;
            if (cudaDeviceGetAttribute(&sl.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PM_ERR_CUDA;
            sl.acc = (unsigned long long*)a;
            sl.flag = (int*)f;
            sl.ready = true;
        }
        slot = sl;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t cells = (size_t)n * n * n;
    // the array keeps the previous call's contents: clear the part this call uses
    if (cudaMemsetAsync(slot.acc, 0, cells * sizeof(unsigned long long), s) != cudaSuccess) return PM_ERR_CUDA;
    if (cudaMemsetAsync(slot.flag, 0, sizeof(int), s) != cudaSuccess) return PM_ERR_CUDA;
    // each launch is checked at once, so that a failure is reported by the call that made it
    launch_deposit_on(s, slot.sms, pos, np, n, slot.acc);
    if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
    launch_density_on(s, slot.sms, (const long long*)slot.acc, n, np, delta, slot.flag);
    if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
    int hflag = 0;
    if (cudaMemcpyAsync(&hflag, slot.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PM_ERR_CUDA;
    return hflag ? PM_ERR_OVERFLOW : PM_OK;
}
