// noalloc.cu -- chunk encode that allocates no device memory.
//
// For callers that cannot allocate GPU memory while they run (device memory
// already owned by another allocator, or loops that cannot absorb the
// device-wide synchronisation of cudaMalloc / cudaFree). The encoder's
// staging -- packed-block slots, per-block sums of q^2, the chunk record and
// the error word -- lives in one file-scope device array instead of buffers
// allocated per call. The array is part of the module image: every GPU that
// loads the library holds it until the process exits.
//
// In host code the array's name denotes a host-side stand-in, not a device
// address, so the device address is looked up with cudaGetSymbolAddress once
// per device (with that device current) and passed to the kernels.
#include <cmath>
#include <mutex>

#include "sv.h"
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kMaxC = SV_NOALLOC_MAX_CHUNK_QUBITS;
constexpr size_t kSparseBytes = (size_t)1 << (kMaxC + 3);        // 1 KiB per 256-value block, both planes
constexpr size_t kBlocksqBytes = (size_t)8 << (kMaxC - 8);       // one u64 per 256-amplitude block pair
constexpr size_t kTailBytes = 256;                               // chunk record + error word
constexpr size_t kScratchBytes = kSparseBytes + kBlocksqBytes + kTailBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the staging array on the current device (set-up on first use).
int scratch_for_current_device(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SV_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return SV_OK;
}

}  // namespace
}  // namespace sv

extern "C" int sv_codec_encode_noalloc(int dtype, int c, double eb, const void* d_amps, void* d_stream, size_t cap,
                                       size_t* h_nbytes)
{
    using namespace sv;
    if ((dtype != SV_C64 && dtype != SV_C128) || c < 8 || c > kMaxC || !d_amps || !d_stream || !h_nbytes)
        return SV_ERR_ARG;
    if (!(eb > 0) || !(eb <= 1.0)) return SV_ERR_ARG;
    int e2 = 0;
    frexp(2.0 * eb, &e2);
    const int k = e2 - 1;  // step 2^k, the largest power of two <= 2 eb
    if (k < -60) return SV_ERR_RANGE;
    const CodecLayout L = codec_layout(c);
    if (cap < L.max_bytes) return SV_ERR_ARG;

    unsigned char* base = nullptr;
    int r = scratch_for_current_device(&base);
    if (r) return r;
    uint32_t* sparse = reinterpret_cast<uint32_t*>(base);
    unsigned long long* blocksq = reinterpret_cast<unsigned long long*>(base + kSparseBytes);
    ChunkOut* co = reinterpret_cast<ChunkOut*>(base + kSparseBytes + kBlocksqBytes);
    int* err = reinterpret_cast<int*>(base + kSparseBytes + kBlocksqBytes + sizeof(ChunkOut));

    // the error word keeps the previous call's value: clear it first
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), 0);
    if (e != cudaSuccess) return SV_ERR_CUDA;
    e = dtype == SV_C64 ? launch_encode<float>(d_amps, c, dtype, k, 1, static_cast<uint8_t*>(d_stream), L.max_bytes,
                                               sparse, blocksq, co, err, 0, nullptr)
                        : launch_encode<double>(d_amps, c, dtype, k, 1, static_cast<uint8_t*>(d_stream), L.max_bytes,
                                                sparse, blocksq, co, err, 0, nullptr);
    if (e != cudaSuccess) return SV_ERR_CUDA;
    ChunkOut hco{};
    int herr = 0;
    if (cudaMemcpy(&hco, co, sizeof(hco), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SV_ERR_CUDA;
    if (herr & kErrRange) return SV_ERR_RANGE;
    *h_nbytes = hco.bytes;
    return SV_OK;
}
