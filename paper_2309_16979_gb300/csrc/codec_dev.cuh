// codec_dev.cuh -- warp-level decode / encode of one 256-amplitude block pair
// (the real-part block and the imaginary-part block of the same amplitudes),
// shared by the stand-alone codec kernels (codec.cu) and the fused tile
// kernels (apply_phase.cu). Stream format: include/sv.h.
//
// Lane `lane` owns amplitudes 8*lane .. 8*lane+7 of the pair. The step is a
// power of two, so x * 2^-k and q * 2^k are exact in the amplitude's own
// precision (no FP64 on the complex64 path).
#pragma once

#include "sv_dev_types.h"

namespace sv {
namespace codec {

constexpr unsigned FULL = 0xffffffffu;

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

template <typename R> __device__ __forceinline__ R pow2(int e);
template <> __device__ __forceinline__ float pow2<float>(int e) { return __int_as_float((127 + e) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int e)
{
    return __longlong_as_double((long long)(1023 + e) << 52);
}

template <typename R> __device__ __forceinline__ int32_t round_q(R y);
template <> __device__ __forceinline__ int32_t round_q<float>(float y) { return __float2int_rn(y); }
template <> __device__ __forceinline__ int32_t round_q<double>(double y) { return __double2int_rn(y); }

template <typename R> __device__ __forceinline__ R from_q(int32_t q);
template <> __device__ __forceinline__ float from_q<float>(int32_t q) { return __int2float_rn(q); }
template <> __device__ __forceinline__ double from_q<double>(int32_t q) { return (double)q; }

template <typename R> struct QLimit;
template <> struct QLimit<float> { static constexpr float v = 16777215.0f; };     // 2^24 - 1
template <> struct QLimit<double> { static constexpr double v = 1073741823.0; };  // 2^30 - 1

// Decoding one block pair runs in stages, so that a warp can overlap the
// memory round trips of two pairs: pair_meta (the header and the pair's
// widths, offsets and anchors, one round trip, validated), pair_load (the
// lane's share of the packed words into registers), pair_stage (into the
// warp's shared words), pair_unpack (widths -> residuals -> inclusive scan
// from the anchor -> q * Delta).
struct PairMeta {
    uint32_t w[2], off[2];
    int32_t anc[2];
    int k;
    bool ok;
};

// block pair bp of the chunk stream s (nbytes long, at most `limit` bytes may
// be read); ok = false (for the whole warp) when the stream fails validation
__device__ __forceinline__ PairMeta pair_meta(const uint8_t* __restrict__ s, uint64_t nbytes, uint64_t limit, int c,
                                              int dtype, uint32_t bp)
{
    PairMeta pm;
    pm.ok = false;
    pm.k = 0;
    for (int p = 0; p < 2; p++) pm.w[p] = pm.off[p] = 0, pm.anc[p] = 0;
    const CodecLayout L = codec_layout(c);
    if (!(nbytes >= L.p_off && nbytes <= limit)) return pm;
    // the header and this pair's metadata lie below p_off <= nbytes: all of
    // them are loaded at once, then validated
    const uint32_t h0 = ld32(s), h1 = ld32(s + 4), nbh = ld32(s + 12);
    const int k = (int32_t)ld32(s + 8);
    const uint32_t total = ld32(s + 16);
    uint32_t nxt[2];
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const uint32_t b = p ? bp + L.bpc : bp;
        pm.w[p] = s[L.w_off + b];
        pm.off[p] = ld32(s + L.o_off + 4ull * b);
        nxt[p] = ld32(s + L.o_off + 4ull * (b + 1));
        pm.anc[p] = (int32_t)ld32(s + L.a_off + 4ull * b);
    }
    bool ok = h0 == kMagic && (h1 & 0xffffu) == 1u && ((h1 >> 16) & 0xffu) == (uint32_t)dtype &&
              (h1 >> 24) == (uint32_t)c && k <= 0 && k >= -60 && nbh == L.nb && L.p_off + 4ull * total <= nbytes;
#pragma unroll
    for (int p = 0; p < 2; p++)
        ok = ok && pm.w[p] <= 32u && nxt[p] - pm.off[p] == 8u * pm.w[p] &&
             L.p_off + 4ull * ((uint64_t)pm.off[p] + 8ull * pm.w[p]) <= nbytes;
    if (bp == 0) ok = ok && ld32(s + L.o_off) == 0u && ld32(s + L.o_off + 4ull * L.nb) == total;
    pm.k = k;
    pm.ok = ok;
    return pm;
}

// the lane's 16-byte words of each plane's packed block (2w <= 64 words)
__device__ __forceinline__ void pair_load(const uint8_t* __restrict__ s, int c, const PairMeta& pm, uint4 (&v)[2][2],
                                          int lane)
{
    const CodecLayout L = codec_layout(c);
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const uint4* src = reinterpret_cast<const uint4*>(s + L.p_off + 4ull * pm.off[p]);
        if ((uint32_t)lane < 2 * pm.w[p]) v[p][0] = src[lane];
        if ((uint32_t)lane + 32 < 2 * pm.w[p]) v[p][1] = src[lane + 32];
    }
}

__device__ __forceinline__ void pair_stage(const PairMeta& pm, const uint4 (&v)[2][2], uint32_t (*sbuf)[264], int lane)
{
#pragma unroll
    for (int p = 0; p < 2; p++) {
        uint4* dst = reinterpret_cast<uint4*>(sbuf[p]);
        if ((uint32_t)lane < 2 * pm.w[p]) dst[lane] = v[p][0];
        if ((uint32_t)lane + 32 < 2 * pm.w[p]) dst[lane + 32] = v[p][1];
        if (lane == 0) sbuf[p][8 * pm.w[p]] = 0u;
    }
}

// x[plane][m] for j = 8*lane + m from the staged words (after a __syncwarp)
template <typename R>
__device__ __forceinline__ void pair_unpack(const PairMeta& pm, const uint32_t (*sbuf)[264], R scale, R (&x)[2][8],
                                            int lane)
{
    const R delta = pow2<R>(pm.k);
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const uint32_t ww = pm.w[p];
        const uint32_t mask = ww >= 32u ? FULL : ((1u << ww) - 1u);
        uint32_t v[8];
        // the lane's 8 values are its 8 ww consecutive bits from bit 8 lane ww:
        // read word by word into a 64-bit accumulator as they are needed
        const uint32_t pos = 8u * (uint32_t)lane * ww;
        uint32_t wi = pos >> 5;
        uint64_t acc = ww ? (uint64_t)(sbuf[p][wi] >> (pos & 31)) : 0ull;
        uint32_t nb = 32u - (pos & 31);
        wi++;
#pragma unroll
        for (int m = 0; m < 8; m++) {
            const uint32_t j = 8u * lane + m;
            if (nb < ww) {
                acc |= (uint64_t)sbuf[p][wi] << nb;
                nb += 32u;
                wi++;
            }
            const uint32_t z = (uint32_t)acc & mask;
            acc >>= ww;
            nb -= ww;
            const uint32_t rr = (z >> 1) ^ (0u - (z & 1u));
            v[m] = (j == 0) ? 0u : rr;
        }
#pragma unroll
        for (int m = 1; m < 8; m++) v[m] += v[m - 1];
        const uint32_t tot = v[7];
        uint32_t incl = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t base = (uint32_t)pm.anc[p] + (incl - tot);
#pragma unroll
        for (int m = 0; m < 8; m++) {
            R val = from_q<R>((int32_t)(base + v[m])) * delta;
            if (scale != (R)1) val *= scale;
            x[p][m] = val;
        }
    }
}

// Validate and decode block pair bp of the chunk stream s (nbytes long, at
// most `limit` bytes may be read) into x[plane][m] for j = 8*lane + m.
// sbuf: this warp's 2 x 264 words of shared memory. Returns false (for the
// whole warp) if the stream fails validation; x is then undefined.
template <typename R>
__device__ __forceinline__ bool decode_pair(const uint8_t* __restrict__ s, uint64_t nbytes, uint64_t limit, int c,
                                            int dtype, uint32_t bp, uint32_t (*sbuf)[264], R scale, R (&x)[2][8],
                                            int lane)
{
    const PairMeta pm = pair_meta(s, nbytes, limit, c, dtype, bp);
    if (!pm.ok) return false;
    uint4 v[2][2];
    pair_load(s, c, pm, v, lane);
    __syncwarp();
    pair_stage(pm, v, sbuf, lane);
    __syncwarp();
    pair_unpack<R>(pm, sbuf, scale, x, lane);
    return true;
}

// Encode x[plane][m] (j = 8*lane + m) as block pair bp of a chunk whose output
// stream starts at so: width and anchor go to the stream's metadata, the
// packed words to the chunk's staging slots (1 KiB per block), the pair's
// sum of q^2 to *blocksq. pk: this warp's 2 x 260 words of shared memory.
template <typename R>
__device__ __forceinline__ void encode_pair(const R (&x)[2][8], int c, int k, uint32_t bp, uint8_t* __restrict__ so,
                                            uint32_t* __restrict__ sparse_chunk,
                                            unsigned long long* __restrict__ blocksq, uint32_t (*pk)[260],
                                            int* err, int lane)
{
    const CodecLayout L = codec_layout(c);
    const R inv = pow2<R>(-k);
    const R qmax = QLimit<R>::v;
    int32_t q[2][8];
    bool bad = false;
    unsigned long long ss = 0;
#pragma unroll
    for (int p = 0; p < 2; p++) {
#pragma unroll
        for (int m = 0; m < 8; m++) {
            R y = x[p][m] * inv;  // exact: inv is a power of two
            if (!(fabs(y) <= qmax)) { bad = true; y = (R)0; }
            q[p][m] = round_q<R>(y);
            ss += (unsigned long long)((long long)q[p][m] * (long long)q[p][m]);
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, kErrRange);
    uint32_t wpl[2];
    int32_t anchor[2];
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int32_t prev = __shfl_up_sync(FULL, q[p][7], 1);
        uint32_t z[8], mx = 0;
#pragma unroll
        for (int m = 0; m < 8; m++) {
            int32_t rr;
            if (m == 0) rr = (lane == 0) ? 0 : q[p][0] - prev;
            else rr = q[p][m] - q[p][m - 1];
            z[m] = ((uint32_t)rr << 1) ^ (uint32_t)(rr >> 31);
            mx = max(mx, z[m]);
        }
        mx = __reduce_max_sync(FULL, mx);
        const uint32_t w = mx ? 32u - (uint32_t)__clz(mx) : 0u;
        // value j = 8 lane + m takes bits [j w, (j + 1) w) of the block's words
        if (w >= 4) {
            // a lane's 8 w >= 32 bits complete at least one word: it packs them
            // in a 64-bit accumulator and stores each word it completes; its
            // first word's low bits (when it starts inside a word) belong to
            // the previous lane, whose leftover (the accumulator's final
            // partial word) is shuffled up and OR-ed in after the stores
            const uint32_t pos = 8u * (uint32_t)lane * w;
            uint32_t wi = pos >> 5, nb = pos & 31;
            uint64_t acc = 0;
#pragma unroll
            for (int m = 0; m < 8; m++) {
                acc |= (uint64_t)z[m] << nb;
                nb += w;
                if (nb >= 32u) {
                    pk[p][wi] = (uint32_t)acc;
                    acc >>= 32;
                    nb -= 32u;
                    wi++;
                }
            }
            // lane 31 ends on the block's last bit (256 w is a multiple of 32)
            const uint32_t prev = __shfl_up_sync(FULL, (uint32_t)acc, 1);
            __syncwarp();
            if (lane > 0 && (pos & 31)) pk[p][pos >> 5] |= prev;
        } else if (w) {
            // fewer than 32 bits a lane: words shared by several lanes
            for (uint32_t i = (uint32_t)lane; i <= 8u * w; i += 32) pk[p][i] = 0u;
            __syncwarp();
#pragma unroll
            for (int m = 0; m < 8; m++) {
                const uint32_t pos = (8u * lane + m) * w;
                const uint32_t wi = pos >> 5, bit = pos & 31;
                atomicOr(&pk[p][wi], z[m] << bit);
                if (bit + w > 32u) atomicOr(&pk[p][wi + 1], z[m] >> (32u - bit));
            }
        }
        wpl[p] = w;
        anchor[p] = __shfl_sync(FULL, q[p][0], 0);
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const uint32_t b = p ? bp + L.bpc : bp;
        const uint32_t w = wpl[p];
        uint4* dst = reinterpret_cast<uint4*>(sparse_chunk + (uint64_t)b * 256ull);
        const uint4* srcv = reinterpret_cast<const uint4*>(pk[p]);
        for (uint32_t i = lane; i < 2 * w; i += 32) dst[i] = srcv[i];
        if (lane == 0) {
            so[L.w_off + b] = (uint8_t)w;
            *reinterpret_cast<int32_t*>(so + L.a_off + 4ull * b) = anchor[p];
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) ss += __shfl_down_sync(FULL, ss, d);
    if (lane == 0) *blocksq = ss;
}

}  // namespace codec
}  // namespace sv
