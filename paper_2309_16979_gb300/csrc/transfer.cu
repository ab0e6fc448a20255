// transfer.cu -- the three ways of moving a state vector between host and
// device memory that the paper compares (Sec. 2 "Online stage", step (2),
// and Table 1): one bulk copy in index order ("sync"), one asynchronous copy per amplitude
// straight to its position ("async"), and one bulk copy into a device
// staging buffer followed by a kernel that moves every amplitude to its
// position ("buffer"; the reverse order for device to host).
//
// The positions: amplitude i of the host array belongs at index remap(i) of
// the device state, i with the low n/2 and the high n - n/2 bits of its index
// exchanged (a chunk's amplitudes end up strided, as when a chunk joins a
// staged group whose staged qubits are not its top bits).
#include <chrono>
#include <cstring>

#include "sv.h"
#include "sv_internal.h"

namespace sv {
namespace {

__host__ __device__ inline uint64_t remap_index(uint64_t i, int n)
{
    const int h = n / 2;
    return (i >> h) | ((i & ((1ull << h) - 1)) << (n - h));
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ src, T* __restrict__ dst, int n)
{
    const uint64_t count = 1ull << n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        dst[remap_index(i, n)] = src[i];
}

template <typename T>
__global__ void k_gather(const T* __restrict__ src, T* __restrict__ dst, int n)
{
    const uint64_t count = 1ull << n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[remap_index(i, n)];
}

// amplitude i of the pattern: (i, -i) in the amplitude's type
template <typename T>
void fill_pattern(T* h, uint64_t count)
{
    for (uint64_t i = 0; i < count; i++) {
        h[i].x = (decltype(h[i].x))i;
        h[i].y = -(decltype(h[i].y))i;
    }
}

template <typename T>
int probe(int n, int strategy, int direction, uint64_t sample, double* seconds, int* verified)
{
    const uint64_t count = 1ull << n, bytes = count * sizeof(T);
    if (sample == 0 || sample > count) sample = count;
    T *h = nullptr, *d = nullptr, *b = nullptr, *chk = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e;
    int r = SV_OK;
    if ((e = cudaHostAlloc(&h, bytes, cudaHostAllocDefault))) {
        cudaGetLastError();
        return SV_ERR_HOST_OOM;
    }
    if ((e = cudaMalloc(&d, bytes)) || (strategy == SV_COPY_BUFFER && (e = cudaMalloc(&b, bytes)))) {
        cudaGetLastError();
        cudaFreeHost(h);
        cudaFree(d);
        return SV_ERR_DEVICE_OOM;
    }
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) r = SV_ERR_CUDA;
    const unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, 152ull * 16);
    // the bulk copy keeps the order (the minimum time to move the bytes); the
    // other two strategies place host amplitude i at device index remap(i)
    const bool placed = strategy != SV_COPY_SYNC;
    // the source side holds the pattern in host order (H2D) or already at the
    // device positions (D2H)
    if (!r) {
        fill_pattern(h, count);
        if (direction == SV_COPY_D2H) {
            T* tmp = nullptr;
            if (cudaMalloc(&tmp, bytes) || cudaMemcpy(placed ? tmp : d, h, bytes, cudaMemcpyHostToDevice))
                r = SV_ERR_CUDA;
            if (!r && placed) {
                k_scatter<T><<<grid, 256, 0, st>>>(tmp, d, n);
                if (cudaStreamSynchronize(st)) r = SV_ERR_CUDA;
            }
            cudaFree(tmp);
            std::memset(h, 0, bytes);
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    if (!r) {
        if (strategy == SV_COPY_SYNC) {
            e = direction == SV_COPY_H2D ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice)
                                         : cudaMemcpy(h, d, bytes, cudaMemcpyDeviceToHost);
        } else if (strategy == SV_COPY_ASYNC) {
            e = cudaSuccess;
            for (uint64_t i = 0; i < sample && !e; i++) {
                const uint64_t p = remap_index(i, n);
                e = direction == SV_COPY_H2D ? cudaMemcpyAsync(d + p, h + i, sizeof(T), cudaMemcpyHostToDevice, st)
                                             : cudaMemcpyAsync(h + i, d + p, sizeof(T), cudaMemcpyDeviceToHost, st);
            }
            if (!e) e = cudaStreamSynchronize(st);
        } else {
            if (direction == SV_COPY_H2D) {
                e = cudaMemcpyAsync(b, h, bytes, cudaMemcpyHostToDevice, st);
                if (!e) k_scatter<T><<<grid, 256, 0, st>>>(b, d, n);
            } else {
                k_gather<T><<<grid, 256, 0, st>>>(d, b, n);
                e = cudaMemcpyAsync(h, b, bytes, cudaMemcpyDeviceToHost, st);
            }
            if (!e) e = cudaStreamSynchronize(st);
        }
        if (e) r = SV_ERR_CUDA;
    }
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!r) {
        // the asynchronous copies were timed on a sample: linear in the count
        *seconds = strategy == SV_COPY_ASYNC ? dt * (double)count / (double)sample : dt;
        // every moved amplitude is where it belongs
        const uint64_t n_check = strategy == SV_COPY_ASYNC ? sample : count;
        bool ok = true;
        if (direction == SV_COPY_H2D) {
            if (cudaHostAlloc(&chk, bytes, cudaHostAllocDefault) || cudaMemcpy(chk, d, bytes, cudaMemcpyDeviceToHost)) {
                r = SV_ERR_CUDA;
            } else {
                for (uint64_t i = 0; i < n_check && ok; i++) {
                    const T v = chk[placed ? remap_index(i, n) : i];
                    ok = v.x == (decltype(v.x))i && v.y == -(decltype(v.y))i;
                }
            }
        } else {
            for (uint64_t i = 0; i < n_check && ok; i++) ok = h[i].x == (decltype(h[i].x))i && h[i].y == -(decltype(h[i].y))i;
        }
        if (verified) *verified = ok ? 1 : 0;
    }
    if (st) cudaStreamDestroy(st);
    cudaFreeHost(h);
    if (chk) cudaFreeHost(chk);
    cudaFree(d);
    cudaFree(b);
    return r;
}

}  // namespace
}  // namespace sv

extern "C" int sv_copy_probe(int n, int dtype, int strategy, int direction, uint64_t sample, double* seconds,
                             int* verified)
{
    if (n < 1 || n > 34 || (dtype != SV_C64 && dtype != SV_C128) || !seconds ||
        (strategy != SV_COPY_SYNC && strategy != SV_COPY_ASYNC && strategy != SV_COPY_BUFFER) ||
        (direction != SV_COPY_H2D && direction != SV_COPY_D2H))
        return SV_ERR_ARG;
    return dtype == SV_C64 ? sv::probe<float2>(n, strategy, direction, sample, seconds, verified)
                           : sv::probe<double2>(n, strategy, direction, sample, seconds, verified);
}
