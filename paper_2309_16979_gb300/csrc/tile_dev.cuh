// tile_dev.cuh -- tile staging shared by the register-phase kernel
// (apply_phase.cu) and the sub-pass kernels generated at run time (jit.cpp):
// the shared-memory swizzle, the per-CTA row table, HBM <-> shared copies of
// one 2^12-amplitude tile, and the fused codec steps that replace them.
//
// Two shared-memory layouts of a tile keep the 16 lanes of a half-warp, whose
// four low thread bits map to tile bits of four different residues mod 4, on
// 16 different bank pairs whatever the register qubits are:
//  - SwzLayout: amplitude i at swz(i) = i ^ (((i >> 4) ^ (i >> 8)) & 15),
//    linear over XOR (a register's address is the thread's base XOR a
//    constant);
//  - PadLayout: amplitude i at i + (i >> 4) + (i >> 8) (a spare slot after
//    every 16 and every 256 amplitudes), additive over disjoint bit sets (a
//    register's address is the thread's base plus a constant, folded into
//    the load's immediate offset). Tile bit b moves the slot by 2^(b mod 4)
//    modulo 16 in both.
#pragma once

#include "codec_dev.cuh"

namespace sv {
namespace tile {

constexpr int kThreads = 256;
constexpr int kT = kPhaseTileQubits;  // 12
constexpr int kN = 1 << kT;           // 4096 amplitudes per tile
constexpr int kMinLowBits = kTileLowQubits;  // rows of at least 16 contiguous amplitudes
constexpr int kCodecWords = 2 * 264;  // per-warp codec staging (decode payload / encode packing)

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15u); }

template <typename T, typename R>
__device__ __forceinline__ T mk2(R x, R y)
{
    T v;
    v.x = x;
    v.y = y;
    return v;
}

// at(a | b) = join(at(a), at(b)) for offsets a, b with disjoint bits
struct SwzLayout {
    static __device__ __forceinline__ uint32_t at(uint32_t i) { return swz(i); }
    static __device__ __forceinline__ uint32_t join(uint32_t a, uint32_t b) { return a ^ b; }
};

struct PadLayout {
    static __device__ __forceinline__ uint32_t at(uint32_t i) { return i + (i >> 4) + (i >> 8); }
    static __device__ __forceinline__ uint32_t join(uint32_t a, uint32_t b) { return a + b; }
};
// slots of one padded tile buffer: the last slot + 1, rounded up to 16 (a
// second buffer stays 16-byte aligned); jit.cpp sizes shared memory the same way
constexpr uint32_t kPadElems = ((kN - 1) + (kN - 1) / 16 + (kN - 1) / 256 + 1 + 15) & ~15u;
static_assert(kPadElems == 4368, "padded tile buffer");

// Per-CTA tables: local offset of each tile row, and the local offset of
// each 4-bit digit of a tile index (tile index bit i -> local bit opos[i];
// digit k covers index bits 4k..4k+3).
constexpr int kBaseDigits = (kMaxLocalQubits - kT + 3) / 4;
struct Rows {
    uint64_t rowoff[1 << (kT - kMinLowBits)];
    uint64_t digit[kBaseDigits][16];
};

__device__ __forceinline__ void setup_rows(Rows& rt, const TileDesc& td)
{
    const uint32_t nrows = 1u << (kT - td.l);
    for (uint32_t rw = threadIdx.x; rw < nrows; rw += blockDim.x) {
        uint64_t off = 0;
        for (int i = 0; i < kT - td.l; i++)
            if ((rw >> i) & 1u) off |= 1ull << td.hpos[i];
        rt.rowoff[rw] = off;
    }
    for (int e = threadIdx.x; e < 16 * ((td.nout + 3) >> 2); e += blockDim.x) {
        const int k = e >> 4;
        uint64_t off = 0;
        for (int b = 0; b < 4; b++)
            if (((e >> b) & 1) && 4 * k + b < td.nout) off |= 1ull << td.opos[4 * k + b];
        rt.digit[k][e & 15] = off;
    }
}

// local offset of tile `tile`: the offsets of its 4-bit digits
__device__ __forceinline__ uint64_t tile_base(const Rows& rt, const TileDesc& td, uint64_t tile)
{
    uint64_t base = 0;
    for (int k = 0; k < ((td.nout + 3) >> 2); k++) base |= rt.digit[k][(tile >> (4 * k)) & 15];
    return base;
}

// Fused codec steps, out of line: they run once per row, not per gate.
template <typename T, typename R, typename Lay = SwzLayout>
__device__ __noinline__ void decode_row(T* s, uint32_t rw, const FuseArgs& fa, uint64_t li, uint32_t* cw, int lane)
{
    const uint64_t cmask = (1ull << fa.c) - 1;
    const uint32_t r = (uint32_t)(li >> fa.c);
    const uint32_t bp = (uint32_t)((li & cmask) >> 8);
    R x[2][8];
    if (!codec::decode_pair<R>(fa.in + (size_t)r * fa.in_stride, fa.gin.bytes[r], fa.in_stride, fa.c, fa.dtype, bp,
                               reinterpret_cast<uint32_t(*)[264]>(cw), (R)fa.scale, x, lane)) {
        if (lane == 0) atomicOr(fa.err, kErrCorrupt);
#pragma unroll
        for (int m = 0; m < 8; m++) x[0][m] = x[1][m] = (R)0;
    }
#pragma unroll
    for (int m = 0; m < 8; m++) {
        T v;
        v.x = x[0][m];
        v.y = x[1][m];
        s[Lay::at(rw * 256u + 8u * lane + m)] = v;
    }
}

template <typename T, typename R, typename Lay = SwzLayout>
__device__ __noinline__ void encode_row(const T* s, uint32_t rw, const FuseArgs& fa, uint64_t li, uint32_t* cw,
                                        int lane)
{
    const CodecLayout CL = codec_layout(fa.c);
    const uint64_t cmask = (1ull << fa.c) - 1;
    const uint32_t r = (uint32_t)(li >> fa.c);
    const uint32_t bp = (uint32_t)((li & cmask) >> 8);
    R x[2][8];
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const T v = s[Lay::at(rw * 256u + 8u * lane + m)];
        x[0][m] = v.x;
        x[1][m] = v.y;
    }
    codec::encode_pair<R>(x, fa.c, fa.k, bp, fa.out + (size_t)r * fa.out_stride,
                          fa.sparse + (uint64_t)r * CL.nb * 256ull, fa.blocksq + (uint64_t)r * CL.bpc + bp,
                          reinterpret_cast<uint32_t(*)[260]>(cw), fa.err, lane);
}

// Plain copies of one tile between HBM and shared memory (no codec).
// LB >= 0: the tile's low bits l known at compile time (td.l otherwise).
template <typename T, typename R, typename Lay, int LB = -1>
__device__ __forceinline__ void load_plain(T* s, const T* __restrict__ amps, const Rows& rt, const TileDesc& td,
                                           uint64_t base)
{
    const int l = LB >= 0 ? LB : td.l;
    const uint32_t t2 = 2 * threadIdx.x, rmask = (1u << l) - 1u;
    const T* g0 = amps + base + (t2 & rmask);
    const uint32_t a0 = Lay::at(t2), a1 = Lay::at(t2 + 1);
#pragma unroll
    for (uint32_t k = 0; k < kN / (2 * kThreads); k++) {
        const T* g = g0 + rt.rowoff[(t2 >> l) + ((512u * k) >> l)];
        const uint32_t ak = Lay::at(512u * k);
        T x0, x1;
        if (sizeof(R) == 4) {
            const float4 v = *reinterpret_cast<const float4*>(g);
            x0.x = v.x; x0.y = v.y; x1.x = v.z; x1.y = v.w;
        } else {
            x0 = g[0];
            x1 = g[1];
        }
        s[Lay::join(a0, ak)] = x0;
        s[Lay::join(a1, ak)] = x1;
    }
}

template <typename T, typename R, typename Lay, int LB = -1>
__device__ __forceinline__ void store_plain(const T* s, T* __restrict__ amps, const Rows& rt, const TileDesc& td,
                                            uint64_t base)
{
    const int l = LB >= 0 ? LB : td.l;
    const uint32_t t2 = 2 * threadIdx.x, rmask = (1u << l) - 1u;
    T* g0 = amps + base + (t2 & rmask);
    const uint32_t a0 = Lay::at(t2), a1 = Lay::at(t2 + 1);
#pragma unroll
    for (uint32_t k = 0; k < kN / (2 * kThreads); k++) {
        T* g = g0 + rt.rowoff[(t2 >> l) + ((512u * k) >> l)];
        const uint32_t ak = Lay::at(512u * k);
        const T x0 = s[Lay::join(a0, ak)], x1 = s[Lay::join(a1, ak)];
        if (sizeof(R) == 4) {
            *reinterpret_cast<float4*>(g) = make_float4((float)x0.x, (float)x0.y, (float)x1.x, (float)x1.y);
        } else {
            g[0] = x0;
            g[1] = x1;
        }
    }
}

// HBM (or the compressed streams) -> shared memory for the tile at `base`.
// DEC: decode the group's chunk streams, one warp per 256-amplitude block
// pair (rows are block pairs, td.l = 8); otherwise 16-byte vector loads along
// the rows.
template <typename T, typename R, bool DEC, typename Lay = SwzLayout, int LB = -1>
__device__ __forceinline__ void load_tile(T* s, const T* __restrict__ amps, const Rows& rt, const TileDesc& td,
                                          uint64_t base, const FuseArgs& fa, uint32_t* cw)
{
    const int l = td.l;
    if (DEC) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const uint32_t nrows = 1u << (kT - l);
        for (uint32_t rw = wid; rw < nrows; rw += kThreads / 32)
            decode_row<T, R, Lay>(s, rw, fa, base + rt.rowoff[rw], cw + wid * kCodecWords, lane);
    } else {
        load_plain<T, R, Lay, LB>(s, amps, rt, td, base);
    }
}

// Asynchronous HBM -> shared copy of the tile at `base` (cp.async, one
// amplitude per copy so that the swizzled destinations need no registers),
// committed as one group; cp_async_wait_all() then __syncthreads() make it
// visible. Used to fetch the next tile while the current one is processed.
template <typename T, typename Lay = SwzLayout, int LB = -1>
__device__ __forceinline__ void prefetch_tile(T* s, const T* __restrict__ amps, const Rows& rt, const TileDesc& td,
                                              uint64_t base)
{
    const int l = LB >= 0 ? LB : td.l;
    // amplitude t + 256k (t = thread): row and slot split as in load_tile
    const uint32_t t = threadIdx.x, rmask = (1u << l) - 1u;
    const T* g0 = amps + base + (t & rmask);
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(s), a0 = Lay::at(t);
#pragma unroll
    for (uint32_t k = 0; k < kN / kThreads; k++) {
        const T* g = g0 + rt.rowoff[(t >> l) + ((256u * k) >> l)];
        const uint32_t d = d0 + (uint32_t)sizeof(T) * Lay::join(a0, Lay::at(256u * k));
        if (sizeof(T) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(g) : "memory");
        else
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(g) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// shared memory -> HBM (or the codec staging when ENC) for the tile at `base`
template <typename T, typename R, bool ENC, typename Lay = SwzLayout, int LB = -1>
__device__ __forceinline__ void store_tile(const T* s, T* __restrict__ amps, const Rows& rt, const TileDesc& td,
                                           uint64_t base, const FuseArgs& fa, uint32_t* cw)
{
    const int l = td.l;
    if (ENC) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const uint32_t nrows = 1u << (kT - l);
        for (uint32_t rw = wid; rw < nrows; rw += kThreads / 32)
            encode_row<T, R, Lay>(s, rw, fa, base + rt.rowoff[rw], cw + wid * kCodecWords, lane);
    } else {
        store_plain<T, R, Lay, LB>(s, amps, rt, td, base);
    }
}

}  // namespace tile
}  // namespace sv
