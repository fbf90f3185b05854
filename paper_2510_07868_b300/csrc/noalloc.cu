// nrrs_split_noalloc: the split-and-compact entry point for callers that must not
// allocate device memory on the call path.
//
// Who needs it: a host program that hands all device memory to its own arena at
// start-up (an engine embedding this library), or a frame loop with a hard deadline:
// cudaMalloc / cudaFree may synchronize the whole device, and such callers cannot
// afford that stall or do not own the allocator.  nrrs_split gets its per-block scratch
// from a pool it allocates on first use; this variant uses a fixed array compiled into
// the library instead, so it never allocates.
//
// The scratch below lives in every GPU that loads the library until the process exits.
// Host code may not use `g_split_scratch` as a device address (on the host it names a
// stand-in object); the device address comes from cudaGetSymbolAddress, taken once
// per device with that device current, on the first call made on that device.  With
// lazy module loading (CUDA's default) that lookup is what loads this file's module on
// the device, which places its code and the array in device memory once; callers that
// cannot take that one-time allocation make a first call at start-up.
#include <cstdio>
#include <mutex>
#include <string>

#include "wavefront.cuh"

using namespace nrrs;

namespace {

// One block handles at most this many parents, so the scratch bounds the queue length.
constexpr long long kNoAllocChunk = 4096;
constexpr int kNoAllocMaxBlocks = 16384;  // => at most 67,108,864 parents per call
constexpr long long kNoAllocMaxN = kNoAllocChunk * kNoAllocMaxBlocks;

struct SplitScratch {
    unsigned long long boff[kNoAllocMaxBlocks];  // exclusive prefix of the block counts
    unsigned long long bcnt[kNoAllocMaxBlocks];  // children requested per block
};

// 256 KiB per device, shared by every call.
static __device__ __align__(256) SplitScratch g_split_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
SplitScratch* g_addr[kMaxDevices] = {};

}  // namespace

namespace nrrs {
// Records the text nrrs_last_error() returns (defined with the other entry points).
nrrs_status record_error(nrrs_status s, const char* msg);
}  // namespace nrrs

extern "C" NRRS_API nrrs_status nrrs_split_noalloc(
    const float* d_q_orig, int64_t n, const float* d_F, const uint32_t* d_pixel,
    const uint32_t* d_sample, const uint32_t* d_lineage, uint32_t depth, uint32_t seed_lo,
    uint32_t seed_hi, uint32_t frame, int64_t cap, uint32_t* d_X, int64_t* d_prefix,
    uint32_t* d_child_parent, uint32_t* d_child_lineage, int64_t* d_total, int64_t* d_dropped,
    void* stream) {
    if (n < 0 || cap < 0 || cap >= (1ll << 31) || !d_F || !d_total || !d_dropped) {
        return record_error(NRRS_ERR_INVALID_ARG, "bad split sizes or NULL outputs");
    }
    if (n > kNoAllocMaxN) {
        return record_error(NRRS_ERR_INVALID_ARG,
                            "n exceeds the fixed scratch of nrrs_split_noalloc (at most 67108864 parents)");
    }
    if (n > 0 && (!d_q_orig || !d_pixel || !d_sample || !d_lineage || !d_X || !d_prefix)) {
        return record_error(NRRS_ERR_INVALID_ARG, "NULL split array");
    }
    if (cap > 0 && (!d_child_parent || !d_child_lineage)) {
        return record_error(NRRS_ERR_INVALID_ARG, "NULL child arrays");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        return record_error(NRRS_ERR_CUDA, "no usable current device");
    }
    SplitScratch* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_split_scratch);
            if (e != cudaSuccess || !p)
                return record_error(NRRS_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e)).c_str());
            g_addr[dev] = static_cast<SplitScratch*>(p);
        }
        scratch = g_addr[dev];
    }
    SplitArrays a{};
    a.q = d_q_orig; a.n = n; a.F = d_F; a.pixel = d_pixel; a.sample = d_sample;
    a.lineage = d_lineage; a.depth = depth; a.key0 = seed_lo; a.key1 = seed_hi ^ frame;
    a.cap = cap; a.X = d_X; a.prefix = reinterpret_cast<long long*>(d_prefix);
    a.child_parent = d_child_parent; a.child_lineage = d_child_lineage;
    a.total = reinterpret_cast<long long*>(d_total);
    a.dropped = reinterpret_cast<long long*>(d_dropped);
    const int grid = n > 0 ? (int)((n + kNoAllocChunk - 1) / kNoAllocChunk) : 1;
    // Every block writes its own count and the scan writes every offset before either
    // is read, so nothing left in the scratch by an earlier call needs clearing.
    launch_split_arrays(a, scratch->bcnt, scratch->boff, grid, (cudaStream_t)stream);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return record_error(NRRS_ERR_CUDA, (std::string("launch: ") + cudaGetErrorString(e)).c_str());
    return NRRS_OK;
}
