// rs_static.cu -- sampling without any device allocation.
//
// rs_sample_static runs the same split-tree and leaf kernels as rs_sample,
// but every byte of scratch it needs lives in one file-scope device array
// that exists from the moment the library is loaded.  It is meant for
// callers that must not allocate device memory on the fly: a serving loop
// whose allocator owns all device memory, a plugin whose host application
// forbids cudaMalloc after start-up, or code that cannot afford the implicit
// device-wide synchronization of cudaMalloc/cudaFree.
//
// Limits (RS_ECAPACITY beyond them): split-tree depth <= kStaticDepth, and
// leaves whose selection exceeds the shared-memory path are handled only up
// to kStaticBigKeys values (device status RS_ECAPACITY otherwise).
//
// The array is shared by every call in the process: calls that overlap on
// the GPU (on different streams or host threads) race and must be avoided.
// The device address and the table are looked up and built once per device
// and kept for the life of the process: after a cudaDeviceReset the array's
// contents are gone, so the entry point must not be used again after one.
#include <mutex>

#include "rs_internal.h"

namespace {

constexpr int kStaticDepth = 16;                                // at most 2^16 leaves
constexpr uint64_t kStaticNodes = 2ull << kStaticDepth;          // heap records 1 .. 2^17 - 1
constexpr uint64_t kStaticBigKeys = 1ull << 16;                  // general-path pool
constexpr uint64_t kTabBytes = rs::kTabWords * sizeof(double);
constexpr uint64_t kStatusBytes = 256;                           // status word, 256-byte slot
constexpr uint64_t kNodeBytes = kStaticNodes * sizeof(rs::NodeRec);
constexpr uint64_t kOvfBytes = (((1ull << kStaticDepth) + 1) * sizeof(uint32_t) + 255) & ~255ull;
// general-path pool: 3 key arrays, 2 index arrays, counts (see big_pool_bytes)
constexpr uint64_t kBigBytes = ((kStaticBigKeys * 32 + (kStaticBigKeys + 1) * 4) + 255) & ~255ull;
constexpr uint64_t kStaticBytes = kTabBytes + kStatusBytes + kNodeBytes + kOvfBytes + kBigBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_base[kMaxDevices] = {};   // device address of g_static_scratch per device

// Once per device, with that device current: look up the array's device
// address (a host-side reference to the symbol is not a device pointer) and
// build the ln i! table in it.
int static_setup(int dev, cudaStream_t st, unsigned char** base) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_base[dev]) {
        *base = g_base[dev];
        return RS_OK;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RS_ECUDA;
    unsigned char* b = static_cast<unsigned char*>(p);
    if (rs::launch_lf_table(reinterpret_cast<double*>(b), st) != cudaSuccess) return RS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RS_ECUDA;
    g_base[dev] = b;
    *base = b;
    return RS_OK;
}

}  // namespace

extern "C" int rs_sample_static(uint64_t n, uint64_t N, uint64_t seed, uint32_t n0, uint64_t* out_dev,
                                void* stream) {
    if (n0 == 0 || N > (1ull << 62) || (n > 0 && N == 0) || n > N) return RS_EINVAL;
    if (n > 0 && (out_dev == nullptr || ((uintptr_t)out_dev & 7))) return RS_EINVAL;
    if (n == 0) return RS_OK;
    const int D = rs::tree_depth(n, N, n0);   // the same depth as rs_sample's
    if (D > kStaticDepth) return RS_ECAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    int rc = static_setup(dev, st, &base);
    if (rc) return rc;
    double* tab = reinterpret_cast<double*>(base);
    int* status = reinterpret_cast<int*>(base + kTabBytes);
    rs::NodeRec* nodes = reinterpret_cast<rs::NodeRec*>(base + kTabBytes + kStatusBytes);
    uint32_t* ovf = reinterpret_cast<uint32_t*>(base + kTabBytes + kStatusBytes + kNodeBytes);
    void* big = base + kTabBytes + kStatusBytes + kNodeBytes + kOvfBytes;
    // The array keeps the previous call's contents: clear the status word
    // (the leaf launch clears the overflow counter itself).
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return RS_ECUDA;
    if (rs::launch_tree(nodes, n, N, seed, D, false, tab, status, st) != cudaSuccess) return RS_ECUDA;
    const uint64_t nleaves = 1ull << D;
    const uint64_t smax = (N >> D) + ((N & (nleaves - 1)) ? 1 : 0);
    const uint64_t bound = std::min<uint64_t>(n, smax - smax / 2);
    rs::LeafLaunch L{};
    L.leaves = nodes + nleaves;
    L.nleaves = nleaves;
    L.first_id = nleaves;
    L.seed = seed;
    L.smax = smax;
    L.out = out_dev;
    L.status = status;
    L.ovf_list = ovf;
    L.ovf_count = ovf + nleaves;
    L.big_pool = big;
    L.big_kmax = bound > 64 ? std::min<uint64_t>(bound, kStaticBigKeys) : 0;
    L.cap = 0;
    L.mean_count = n >> D;   // picks the leaf kernel's shape as rs_sample does (both use shared memory only)
    L.pow2_leaves = (N & (nleaves - 1)) == 0 && (smax & (smax - 1)) == 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RS_ECUDA;
    L.sms = sms;
    L.with_replacement = false;
    if (rs::launch_leaves(L, st) != cudaSuccess) return RS_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RS_ECUDA;
    return h;
}
