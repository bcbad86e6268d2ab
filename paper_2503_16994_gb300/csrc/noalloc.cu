// lqcd_pion_contract_noalloc: the pion contraction for callers that cannot
// allocate device memory.
//
// lqcd_pion_contract needs a lattice handle and keeps its reduction
// scratch in buffers the library allocates with cudaMalloc.  Some callers
// cannot allow that: a process whose device memory is owned by another
// allocator (a framework's caching allocator or a pool sized up front
// holds the free memory, so a cudaMalloc can fail or fragment it), or a
// loop that must not allocate per call because cudaMalloc/cudaFree can
// synchronize the device and stall work queued by others.  This entry
// point allocates nothing: its scratch is a fixed-size array in the
// library's device image, present on every GPU that loads the library
// until the process exits.
#include <mutex>

#include "lqcd_impl.h"

namespace lqcd {

// defined in field_ops.cu
__global__ void contract_aos_kernel(long V, long v3, int T, int src_t, const double *prop, double *partial,
                                    unsigned *counter, double *corr);

// Static scratch: per-slice partial sums and per-slice arrival counters.
constexpr long kNoallocPartials = 1L << 18;  // 262144 doubles = 2 MiB
constexpr int kNoallocSlices = 8192;         // time extent limit
static __device__ __align__(256) double g_noalloc_partial[kNoallocPartials];
static __device__ __align__(256) unsigned g_noalloc_counter[kNoallocSlices];

namespace {
struct ScratchPtrs {
    double *partial = nullptr;
    unsigned *counter = nullptr;
};
std::mutex g_noalloc_mu;
std::map<int, ScratchPtrs> g_noalloc_ptrs;  // per device ordinal

// Device addresses of the static arrays for the current device, looked up
// once per device (host code may not use the symbols' own names as
// device addresses).
int scratch_for_current_device(ScratchPtrs *out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(LQCD_ECUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_ptrs.find(dev);
    if (it != g_noalloc_ptrs.end()) {
        *out = it->second;
        return LQCD_OK;
    }
    ScratchPtrs p;
    cudaError_t e = cudaGetSymbolAddress((void **)&p.partial, g_noalloc_partial);
    if (e != cudaSuccess) return fail(LQCD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress((void **)&p.counter, g_noalloc_counter);
    if (e != cudaSuccess) return fail(LQCD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptrs.emplace(dev, p);
    *out = p;
    return LQCD_OK;
}
}  // namespace

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_pion_contract_noalloc(const int dims[4], const double *prop, int src_t, double *corr,
                                          void *stream)
{
    if (!dims || !prop || !corr) return fail(LQCD_EINVAL, "null argument");
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 1) return fail(LQCD_EINVAL, "every extent must be >= 1");
        V *= dims[m];
    }
    const int T = dims[3];
    if (src_t < 0 || src_t >= T) return fail(LQCD_EINVAL, "source time outside the lattice");
    const long v3 = V / T;
    const long nchunk = (v3 * 12 + kBlock * 4 - 1) / (kBlock * 4);
    if (T > kNoallocSlices || (long)T * nchunk > kNoallocPartials)
        return fail(LQCD_EINVAL, "lattice too large for the static scratch of lqcd_pion_contract_noalloc (needs " +
                                     std::to_string((long)T * nchunk) + " partial sums and " + std::to_string(T) +
                                     " counters; it holds " + std::to_string(kNoallocPartials) + " and " +
                                     std::to_string(kNoallocSlices) + "): use lqcd_pion_contract");
    ScratchPtrs sp;
    if (int rc = scratch_for_current_device(&sp)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counters must start at zero; the partial sums are written before they are read
    cudaError_t e = cudaMemsetAsync(sp.counter, 0, sizeof(unsigned) * T, st);
    if (e != cudaSuccess) return fail(LQCD_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    contract_aos_kernel<<<dim3(unsigned(nchunk), T), kBlock, 0, st>>>(V, v3, T, src_t, prop, sp.partial, sp.counter,
                                                                      corr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LQCD_ECUDA, std::string("contraction launch: ") + cudaGetErrorString(e));
    return LQCD_OK;
}
