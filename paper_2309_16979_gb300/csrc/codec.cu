// codec.cu -- GPU chunk codec (decode / encode) for the compressed store.
//
// MEMQSim (Sec. 2, "Offline stage") compresses each chunk of the state vector
// independently and stores it in CPU memory; the online stage decompresses
// chunks, updates them and recompresses them (steps (1) and (6)). The paper
// names no compressor. This codec is an error-bounded linear quantiser with
// 1-D Lorenzo prediction inside 256-value blocks and fixed-length bit packing
// per block with prefix-sum block offsets; the stream format is documented in
// include/sv.h.
//
// Design for sm_103a:
//   * one warp owns one 256-amplitude block pair (the real-part block and the
//     imaginary-part block of the same amplitudes), so amplitudes are read and
//     written as interleaved complex values with 16-byte vector accesses;
//   * the step is a power of two, so x * 2^-k and q * 2^k are exact in the
//     amplitude's own precision: no FP64 on the complex64 path and no rounding
//     difference to any IEEE implementation;
//   * Lorenzo residuals cross lanes with one shuffle, block widths come from a
//     warp max-reduction, and decode rebuilds q with a warp scan;
//   * packing goes through shared memory (atomicOr of each value's w bits),
//     then 16-byte stores to a per-block staging slot; a one-CTA-per-chunk scan
//     turns widths into offsets, and a compaction kernel moves each block's
//     8*w words to its final offset.
#include <algorithm>

#include "sv_internal.h"
#include "codec_dev.cuh"

namespace sv {
namespace {

using codec::FULL;
template <typename R> using V2 = codec::V2<R>;

// load / store 8 consecutive amplitudes of one lane
__device__ __forceinline__ void load8(const float2* p, float (&x)[2][8])
{
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int h = 0; h < 4; h++) {
        const float4 v = p4[h];
        x[0][2 * h] = v.x; x[1][2 * h] = v.y; x[0][2 * h + 1] = v.z; x[1][2 * h + 1] = v.w;
    }
}
__device__ __forceinline__ void load8(const double2* p, double (&x)[2][8])
{
#pragma unroll
    for (int m = 0; m < 8; m++) { const double2 v = p[m]; x[0][m] = v.x; x[1][m] = v.y; }
}
__device__ __forceinline__ void store8(float2* p, const float (&x)[2][8])
{
    float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int h = 0; h < 4; h++) p4[h] = make_float4(x[0][2 * h], x[1][2 * h], x[0][2 * h + 1], x[1][2 * h + 1]);
}
__device__ __forceinline__ void store8(double2* p, const double (&x)[2][8])
{
#pragma unroll
    for (int m = 0; m < 8; m++) p[m] = make_double2(x[0][m], x[1][m]);
}

// ----------------------------------------------------------------- decode
// one warp per block pair of the group's chunk streams
template <typename R>
__global__ void __launch_bounds__(256)
k_decode(const uint8_t* __restrict__ in, size_t stride, int c, int dtype, uint64_t nwarps, GroupIn gin,
         typename V2<R>::T* __restrict__ amps, R scale, int* err)
{
    __shared__ __align__(16) uint32_t sbuf[8][2][264];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t gw = (uint64_t)blockIdx.x * 8 + wib;
    if (gw >= nwarps) return;
    const int sh = c - 8;
    const uint32_t r = (uint32_t)(gw >> sh);
    const uint32_t bp = (uint32_t)(gw & ((1ull << sh) - 1));
    R x[2][8];
    if (!codec::decode_pair<R>(in + (size_t)r * stride, gin.bytes[r], stride, c, dtype, bp, sbuf[wib], scale, x,
                               lane)) {
        if (lane == 0) atomicOr(err, kErrCorrupt);
        return;
    }
    store8(amps + ((uint64_t)r << c) + 256ull * bp + 8ull * lane, x);
}

// ----------------------------------------------------------------- encode
template <typename R>
__global__ void __launch_bounds__(256)
k_encode_blocks(const typename V2<R>::T* __restrict__ amps, int c, uint64_t nwarps, int k,
                const int32_t* __restrict__ kc, uint8_t* __restrict__ out, size_t stride,
                uint32_t* __restrict__ sparse, unsigned long long* __restrict__ blocksq, int* err)
{
    __shared__ __align__(16) uint32_t pk[8][2][260];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t gw = (uint64_t)blockIdx.x * 8 + wib;
    if (gw >= nwarps) return;
    const CodecLayout L = codec_layout(c);
    const int sh = c - 8;
    const uint32_t r = (uint32_t)(gw >> sh);
    const uint32_t bp = (uint32_t)(gw & ((1ull << sh) - 1));
    R x[2][8];
    load8(amps + ((uint64_t)r << c) + 256ull * bp + 8ull * lane, x);
    codec::encode_pair<R>(x, c, kc ? kc[r] : k, bp, out + (size_t)r * stride, sparse + (uint64_t)r * L.nb * 256ull,
                          blocksq + (uint64_t)r * L.bpc + bp, pk[wib], err, lane);
}

// One CTA per chunk: widths -> offsets (exclusive scan of 8*w), header,
// zeroed padding, and the chunk's record {bytes, sum q^2}.
__global__ void __launch_bounds__(1024)
k_encode_scan(uint8_t* __restrict__ out, size_t stride, int c, int dtype, int k0, const int32_t* __restrict__ kc,
              const unsigned long long* __restrict__ blocksq, ChunkOut* __restrict__ co)
{
    const int k = kc ? kc[blockIdx.x] : k0;
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long qsum[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t r = blockIdx.x;
    uint8_t* so = out + (size_t)r * stride;
    const CodecLayout L = codec_layout(c);
    const uint32_t nb = L.nb;
    const uint32_t per = (nb + 1023) / 1024;
    const uint32_t b0 = min(nb, tid * per), b1 = min(nb, b0 + per);

    uint32_t local = 0;
    for (uint32_t b = b0; b < b1; b++) local += 8u * so[L.w_off + b];
    uint32_t incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t v = wsum[lane], vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, vi, d);
            if (lane >= d) vi += t;
        }
        wsum[lane] = vi - v;  // exclusive prefix of warp totals
    }
    __syncthreads();
    uint32_t run = wsum[wid] + incl - local;
    for (uint32_t b = b0; b < b1; b++) {
        *reinterpret_cast<uint32_t*>(so + L.o_off + 4ull * b) = run;
        run += 8u * so[L.w_off + b];
    }
    if (b1 == nb && b0 < b1) *reinterpret_cast<uint32_t*>(so + L.o_off + 4ull * nb) = run;

    // sum of q^2 over the chunk's block pairs
    const uint32_t bpc = L.bpc, per2 = (bpc + 1023) / 1024;
    const uint32_t p0 = min(bpc, tid * per2), p1 = min(bpc, p0 + per2);
    unsigned long long s2 = 0;
    for (uint32_t b = p0; b < p1; b++) s2 += blocksq[(uint64_t)r * bpc + b];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s2 += __shfl_down_sync(FULL, s2, d);
    if (lane == 0) qsum[wid] = s2;
    __syncthreads();

    if (tid == 0) {
        unsigned long long tot2 = 0;
        for (int i = 0; i < 32; i++) tot2 += qsum[i];
        // total words = offset[nb]
        const uint32_t total = *reinterpret_cast<const uint32_t*>(so + L.o_off + 4ull * nb);
        uint32_t* h = reinterpret_cast<uint32_t*>(so);
        h[0] = kMagic;
        h[1] = 1u | ((uint32_t)dtype << 16) | ((uint32_t)c << 24);
        h[2] = (uint32_t)k;
        h[3] = nb;
        h[4] = total;
        h[5] = h[6] = h[7] = 0u;
        for (size_t i = L.w_off + nb; i < L.a_off; i++) so[i] = 0;
        for (size_t i = L.a_off + 4ull * nb; i < L.o_off; i++) so[i] = 0;
        for (size_t i = L.o_off + 4ull * (nb + 1); i < L.p_off; i++) so[i] = 0;
        co[r].bytes = L.p_off + 4ull * total;
        co[r].sumsq = tot2;
        co[r].k = k;
        co[r].pad = 0;
    }
}

// Move each block's 8*w packed words to payload + offset[b]. One warp per
// kBlocksPerWarp consecutive blocks of a chunk (fewer when the chunk has
// fewer): their widths and offsets are read at once and every payload load
// is in flight before the first store (a warp per block left the copy
// waiting on memory latency).
constexpr int kBlocksPerWarp = 8;

__global__ void __launch_bounds__(256)
k_encode_compact(uint8_t* __restrict__ out, size_t stride, int c, uint64_t nwarps, int lbw,
                 const uint32_t* __restrict__ sparse)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t gw = (uint64_t)blockIdx.x * 8 + wib;
    if (gw >= nwarps) return;
    const CodecLayout L = codec_layout(c);
    const int sh = c - 7 - lbw;  // log2 warps per chunk
    const int nbw = 1 << lbw;    // blocks of this warp
    const uint32_t r = (uint32_t)(gw >> sh);
    const uint32_t b0 = (uint32_t)(gw & ((1ull << sh) - 1)) << lbw;
    uint8_t* so = out + (size_t)r * stride;
    uint32_t wl = 0, ol = 0;
    if (lane < nbw) {
        wl = so[L.w_off + b0 + lane];
        ol = *reinterpret_cast<const uint32_t*>(so + L.o_off + 4ull * (b0 + lane));
    }
    const uint4* src0 = reinterpret_cast<const uint4*>(sparse + ((uint64_t)r * L.nb + b0) * 256ull);
    uint4 v[kBlocksPerWarp][2];
    uint32_t n[kBlocksPerWarp];  // 16-byte words of block k (2w <= 64)
#pragma unroll
    for (int k = 0; k < kBlocksPerWarp; k++) {
        n[k] = 2u * __shfl_sync(FULL, wl, k);
        const uint4* src = src0 + 64 * k;  // the staging slot of a block is 1 KiB
        if (k < nbw && (uint32_t)lane < n[k]) v[k][0] = src[lane];
        if (k < nbw && (uint32_t)lane + 32 < n[k]) v[k][1] = src[lane + 32];
    }
#pragma unroll
    for (int k = 0; k < kBlocksPerWarp; k++) {
        const uint32_t off = __shfl_sync(FULL, ol, k);
        uint4* dst = reinterpret_cast<uint4*>(so + L.p_off + 4ull * off);
        if (k < nbw && (uint32_t)lane < n[k]) dst[lane] = v[k][0];
        if (k < nbw && (uint32_t)lane + 32 < n[k]) dst[lane + 32] = v[k][1];
    }
}

// Relative bound: the largest |re| or |im| of each chunk, as the bits of a
// non-negative float / double (their order is the values' order), merged by
// atomicMax per CTA; grid.y = chunk.
template <typename R>
__global__ void __launch_bounds__(256)
k_chunk_max(const R* __restrict__ comps, int c, unsigned long long* __restrict__ mbits)
{
    const uint64_t n = 2ull << c, r = blockIdx.y;
    const R* x = comps + r * n;
    unsigned long long m = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        // fabs clears the sign bit (a -0.0 would otherwise order above every value)
        const unsigned long long b = sizeof(R) == 4
                                         ? (unsigned long long)__float_as_uint(fabsf((float)x[i]))
                                         : (unsigned long long)__double_as_longlong(fabs((double)x[i]));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&mbits[r], m);
}

// step exponent of each chunk: floor(log2(2 eb m)) clamped to [-60, 0], 0 for
// an all-zero chunk (2 eb exact, one rounded FP64 product, exact exponent)
template <typename R>
__global__ void k_chunk_steps(const unsigned long long* __restrict__ mbits, double two_eb, int nchunks,
                              int32_t* __restrict__ kc)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nchunks) return;
    const double m = sizeof(R) == 4 ? (double)__uint_as_float((unsigned)mbits[r])
                                    : __longlong_as_double((long long)mbits[r]);
    int k = 0;
    if (m > 0) {
        const double v = __dmul_rn(two_eb, m);
        k = v >= 1.0 ? 0 : max(-60, ilogb(v));
    }
    kc[r] = k;
}

template <typename R>
__global__ void k_fill_basis(typename V2<R>::T* amps, uint64_t count, int64_t one_at)
{
    using T = typename V2<R>::T;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        T v;
        v.x = ((int64_t)i == one_at) ? (R)1 : (R)0;
        v.y = (R)0;
        amps[i] = v;
    }
}

inline unsigned blocks_for_warps(uint64_t nwarps) { return (unsigned)((nwarps + 7) / 8); }

}  // namespace

template <typename R>
cudaError_t launch_decode(const uint8_t* in, size_t stride, int c, int dtype, int nchunks,
                          const GroupIn& gin, void* amps, double scale, int* err, cudaStream_t st)
{
    const uint64_t nwarps = (uint64_t)nchunks << (c - 8);
    k_decode<R><<<blocks_for_warps(nwarps), 256, 0, st>>>(
        in, stride, c, dtype, nwarps, gin, static_cast<typename V2<R>::T*>(amps), (R)scale, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_chunk_steps(const void* amps, int c, int nchunks, double eb, unsigned long long* mbits,
                               int32_t* kc, cudaStream_t st, int* launches)
{
    cudaError_t e = cudaMemsetAsync(mbits, 0, sizeof(unsigned long long) * nchunks, st);
    if (e) return e;
    const unsigned bx = (unsigned)std::min<uint64_t>((2ull << c) / 256 / 8 + 1, 4096);
    k_chunk_max<R><<<dim3(bx, (unsigned)nchunks), 256, 0, st>>>(static_cast<const R*>(amps), c, mbits);
    k_chunk_steps<R><<<(nchunks + 255) / 256, 256, 0, st>>>(mbits, 2.0 * eb, nchunks, kc);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_encode(const void* amps, int c, int dtype, int k, int nchunks, uint8_t* out,
                          size_t stride, uint32_t* sparse, unsigned long long* blocksq,
                          ChunkOut* chunk_out, int* err, cudaStream_t st, int* launches, const int32_t* kc)
{
    const uint64_t nw = (uint64_t)nchunks << (c - 8);
    k_encode_blocks<R><<<blocks_for_warps(nw), 256, 0, st>>>(
        static_cast<const typename V2<R>::T*>(amps), c, nw, k, kc, out, stride, sparse, blocksq, err);
    if (launches) *launches += 1;
    return launch_encode_finish(c, dtype, k, nchunks, out, stride, sparse, blocksq, chunk_out, st, launches, kc);
}

cudaError_t launch_encode_finish(int c, int dtype, int k, int nchunks, uint8_t* out, size_t stride,
                                 const uint32_t* sparse, const unsigned long long* blocksq, ChunkOut* chunk_out,
                                 cudaStream_t st, int* launches, const int32_t* kc)
{
    k_encode_scan<<<nchunks, 1024, 0, st>>>(out, stride, c, dtype, k, kc, blocksq, chunk_out);
    // blocks per chunk: 2^(c-7); a warp takes up to kBlocksPerWarp of them
    const int lbw = std::min(3, c - 7);
    const uint64_t nw2 = (uint64_t)nchunks << (c - 7 - lbw);
    k_encode_compact<<<blocks_for_warps(nw2), 256, 0, st>>>(out, stride, c, nw2, lbw, sparse);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

namespace {

// copy `nb` bytes between 16-byte aligned stream slots, blocks of one stream
__device__ __forceinline__ void copy_stream(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint64_t nb)
{
    const uint64_t nv = nb / 16, step = (uint64_t)gridDim.x * blockDim.x;
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += step) d[i] = s[i];
    for (uint64_t i = nv * 16 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += step) dst[i] = src[i];
}

__global__ void k_copy_streams(const uint8_t* __restrict__ src, const ChunkOut* __restrict__ co,
                               uint8_t* __restrict__ dst, uint64_t* __restrict__ bytes, size_t stride)
{
    const int j = blockIdx.y;
    const uint64_t nb = co[j].bytes < stride ? co[j].bytes : stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) bytes[j] = nb;
    copy_stream(src + (size_t)j * stride, dst + (size_t)j * stride, nb);
}

__global__ void k_gather_streams(const uint8_t* __restrict__ src, const uint64_t* __restrict__ bytes,
                                 size_t src_stride, uint8_t* __restrict__ dst, size_t dst_stride, StreamMoves mv)
{
    const int i = blockIdx.y;
    uint64_t nb = bytes[mv.src[i]];
    nb = nb < src_stride ? nb : src_stride;
    nb = nb < dst_stride ? nb : dst_stride;
    copy_stream(src + (size_t)mv.src[i] * src_stride, dst + (size_t)mv.dst[i] * dst_stride, nb);
}

}  // namespace

cudaError_t launch_copy_streams(const uint8_t* src, const ChunkOut* co, uint8_t* dst, uint64_t* bytes, size_t stride,
                                int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_copy_streams<<<dim3(64, n), 256, 0, st>>>(src, co, dst, bytes, stride);
    return cudaGetLastError();
}

cudaError_t launch_gather_streams(const uint8_t* src, const uint64_t* bytes, size_t src_stride, uint8_t* dst,
                                  size_t dst_stride, const StreamMoves& mv, cudaStream_t st)
{
    if (mv.n <= 0) return cudaSuccess;
    if (mv.n > kMaxGroupChunks) return cudaErrorInvalidValue;
    k_gather_streams<<<dim3(64, mv.n), 256, 0, st>>>(src, bytes, src_stride, dst, dst_stride, mv);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fill_basis(void* amps, uint64_t count, int64_t one_at, cudaStream_t st)
{
    const unsigned blocks = (unsigned)std::min<uint64_t>((count + 255) / 256, 152ull * 16);
    k_fill_basis<R><<<blocks, 256, 0, st>>>(static_cast<typename V2<R>::T*>(amps), count, one_at);
    return cudaGetLastError();
}

template cudaError_t launch_decode<float>(const uint8_t*, size_t, int, int, int, const GroupIn&, void*,
                                          double, int*, cudaStream_t);
template cudaError_t launch_decode<double>(const uint8_t*, size_t, int, int, int, const GroupIn&, void*,
                                           double, int*, cudaStream_t);
template cudaError_t launch_encode<float>(const void*, int, int, int, int, uint8_t*, size_t, uint32_t*,
                                          unsigned long long*, ChunkOut*, int*, cudaStream_t, int*, const int32_t*);
template cudaError_t launch_encode<double>(const void*, int, int, int, int, uint8_t*, size_t, uint32_t*,
                                           unsigned long long*, ChunkOut*, int*, cudaStream_t, int*,
                                           const int32_t*);
template cudaError_t launch_chunk_steps<float>(const void*, int, int, double, unsigned long long*, int32_t*,
                                               cudaStream_t, int*);
template cudaError_t launch_chunk_steps<double>(const void*, int, int, double, unsigned long long*, int32_t*,
                                                cudaStream_t, int*);
template cudaError_t launch_fill_basis<float>(void*, uint64_t, int64_t, cudaStream_t);
template cudaError_t launch_fill_basis<double>(void*, uint64_t, int64_t, cudaStream_t);

}  // namespace sv
