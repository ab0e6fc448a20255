// apply_phase.cu -- register-phase gate application on 2^12-amplitude tiles
// (MEMQSim Sec. 2, "Online stage" step (3): the kernel that updates the
// amplitudes of the staged chunks).
//
// One CTA of 256 threads owns one tile of 4096 amplitudes at a time. The tile
// is read from HBM once (16-byte vectors along contiguous rows) into shared
// memory and written back once. In between, the sub-pass's gates run in
// phases: in a phase every thread holds the 16 amplitudes that vary over four
// tile qubits (the phase's register qubits) and applies, in registers, every
// gate whose mixing qubits are among them; the other eight tile bits are the
// thread's index. Controls and diagonal bits on non-register tile bits are
// per-thread constants, those outside the tile per-CTA constants.
//
// Shared memory is XOR-swizzled: amplitude i sits at i ^ (((i >> 4) ^ (i >> 8))
// & 15), so the 16 lanes of a half-warp, whose four low thread bits the host
// maps to tile bits of four different residues mod 4, hit 16 different bank
// pairs whatever the register qubits are.
//
// Common 2x2 gates have cheaper forms: X (pair exchange, no arithmetic),
// real matrices (H, RY, products: 4 multiply-adds per amplitude) and
// [[a, ib], [ic, d]] with real a..d (RX-like), against 8 for a general
// complex matrix; diagonal gates cost one complex product per amplitude.
#include <algorithm>

#include "codec_dev.cuh"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kT = kPhaseTileQubits;  // 12
constexpr int kN = 1 << kT;           // 4096 amplitudes per tile
constexpr int kRegs = 1 << kPhaseRegBits;
constexpr int kPhaseLowBits = 5;

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15u); }

template <typename T, typename R>
__device__ __forceinline__ T cmul(R ar, R ai, T b)
{
    T o;
    o.x = ar * b.x - ai * b.y;
    o.y = ar * b.y + ai * b.x;
    return o;
}

// ---------------------------------------------------- 2x2 forms on bit B
template <int B, typename T, typename R>
__device__ __forceinline__ void d1_generic(T (&a)[kRegs], const R* m, uint32_t rm)
{
    const R m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3], m4 = m[4], m5 = m[5], m6 = m[6], m7 = m[7];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if ((i & rm) != rm) continue;
        const int j = i | (1 << B);
        const T x = a[i], y = a[j];
        T o0, o1;
        o0.x = m0 * x.x - m1 * x.y + m2 * y.x - m3 * y.y;
        o0.y = m0 * x.y + m1 * x.x + m2 * y.y + m3 * y.x;
        o1.x = m4 * x.x - m5 * x.y + m6 * y.x - m7 * y.y;
        o1.y = m4 * x.y + m5 * x.x + m6 * y.y + m7 * y.x;
        a[i] = o0;
        a[j] = o1;
    }
}

template <int B, typename T, typename R>
__device__ __forceinline__ void d1_real(T (&a)[kRegs], const R* m, uint32_t rm)
{
    const R m0 = m[0], m2 = m[2], m4 = m[4], m6 = m[6];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if ((i & rm) != rm) continue;
        const int j = i | (1 << B);
        const T x = a[i], y = a[j];
        T o0, o1;
        o0.x = m0 * x.x + m2 * y.x;
        o0.y = m0 * x.y + m2 * y.y;
        o1.x = m4 * x.x + m6 * y.x;
        o1.y = m4 * x.y + m6 * y.y;
        a[i] = o0;
        a[j] = o1;
    }
}

// [[p, i q], [i r, s]] with real p, q, r, s (m[0] = p, m[3] = q, m[5] = r, m[6] = s)
template <int B, typename T, typename R>
__device__ __forceinline__ void d1_rx(T (&a)[kRegs], const R* m, uint32_t rm)
{
    const R p = m[0], q = m[3], r = m[5], s = m[6];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if ((i & rm) != rm) continue;
        const int j = i | (1 << B);
        const T x = a[i], y = a[j];
        T o0, o1;
        o0.x = p * x.x - q * y.y;
        o0.y = p * x.y + q * y.x;
        o1.x = s * y.x - r * x.y;
        o1.y = s * y.y + r * x.x;
        a[i] = o0;
        a[j] = o1;
    }
}

template <int B, typename T>
__device__ __forceinline__ void d1_swap(T (&a)[kRegs], uint32_t rm)
{
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if ((i & rm) != rm) continue;
        const int j = i | (1 << B);
        const T x = a[i];
        a[i] = a[j];
        a[j] = x;
    }
}

template <int B0, int B1, typename T, typename R>
__device__ __forceinline__ void d2(T (&a)[kRegs], const R* m, uint32_t rm)
{
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & ((1 << B0) | (1 << B1))) continue;
        if ((i & rm) != rm) continue;
        int idx[4];
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            idx[k] = i | ((k & 1) << B0) | (((k >> 1) & 1) << B1);
            v[k] = a[idx[k]];
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            T acc;
            acc.x = (R)0;
            acc.y = (R)0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const R mr = m[2 * (4 * r + k)], mi = m[2 * (4 * r + k) + 1];
                acc.x += mr * v[k].x - mi * v[k].y;
                acc.y += mr * v[k].y + mi * v[k].x;
            }
            a[idx[r]] = acc;
        }
    }
}

template <typename T, typename R>
__device__ __forceinline__ void apply_d1(int type, int r0, T (&a)[kRegs], const R* m, uint32_t rm)
{
#define SV_D1_CASE(B)                                          \
    case B:                                                    \
        if (type == POP_SWAP) d1_swap<B>(a, rm);               \
        else if (type == POP_REAL) d1_real<B>(a, m, rm);       \
        else if (type == POP_RXLIKE) d1_rx<B>(a, m, rm);       \
        else d1_generic<B>(a, m, rm);                          \
        break;
    switch (r0) {
        SV_D1_CASE(0)
        SV_D1_CASE(1)
        SV_D1_CASE(2)
        SV_D1_CASE(3)
        default: break;
    }
#undef SV_D1_CASE
}

template <typename T, typename R>
__device__ __forceinline__ void apply_d2(int r0, int r1, T (&a)[kRegs], const R* m, uint32_t rm)
{
    switch (r0 * 4 + r1) {
        case 1: d2<0, 1>(a, m, rm); break;
        case 2: d2<0, 2>(a, m, rm); break;
        case 3: d2<0, 3>(a, m, rm); break;
        case 4: d2<1, 0>(a, m, rm); break;
        case 6: d2<1, 2>(a, m, rm); break;
        case 7: d2<1, 3>(a, m, rm); break;
        case 8: d2<2, 0>(a, m, rm); break;
        case 9: d2<2, 1>(a, m, rm); break;
        case 11: d2<2, 3>(a, m, rm); break;
        case 12: d2<3, 0>(a, m, rm); break;
        case 13: d2<3, 1>(a, m, rm); break;
        case 14: d2<3, 2>(a, m, rm); break;
        default: break;
    }
}

// constant part of a diagonal source; sets reg_bit (or -1) for register sources
__device__ __forceinline__ uint32_t diag_src(int32_t src, uint32_t tb, uint64_t base, uint64_t gbase, int& reg_bit)
{
    reg_bit = -1;
    if (src < 0) return 0;
    if (src < PSRC_TILE) { reg_bit = src - PSRC_REG; return 0; }
    if (src < PSRC_LOCAL) return (tb >> (src - PSRC_TILE)) & 1u;
    if (src < PSRC_GLOBAL) return (uint32_t)((base >> (src - PSRC_LOCAL)) & 1ull);
    return (uint32_t)((gbase >> (src - PSRC_GLOBAL)) & 1ull);
}

template <typename T, typename R>
__device__ __forceinline__ void apply_diag(const PhaseOp<R>& op, T (&a)[kRegs], uint32_t tb, uint64_t base,
                                           uint64_t gbase, uint32_t rm)
{
    int rb0, rb1;
    const uint32_t c0 = diag_src(op.d0, tb, base, gbase, rb0);
    const uint32_t c1 = diag_src(op.d1, tb, base, gbase, rb1);
    const R e0r = op.m[0], e0i = op.m[1], e1r = op.m[2], e1i = op.m[3];
    const R e2r = op.m[4], e2i = op.m[5], e3r = op.m[6], e3i = op.m[7];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if ((i & rm) != rm) continue;
        const uint32_t b0 = rb0 >= 0 ? ((uint32_t)i >> rb0) & 1u : c0;
        const uint32_t b1 = rb1 >= 0 ? ((uint32_t)i >> rb1) & 1u : c1;
        const uint32_t v = b0 | (b1 << 1);
        const R er = v == 0 ? e0r : v == 1 ? e1r : v == 2 ? e2r : e3r;
        const R ei = v == 0 ? e0i : v == 1 ? e1i : v == 2 ? e2i : e3i;
        a[i] = cmul<T, R>(er, ei, a[i]);
    }
}

// Dynamic shared memory: the tile, then per-warp codec staging (decode
// payload words / encode packing buffer, 2 x 264 words per warp).
constexpr int kCodecWords = 2 * 264;

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_apply_phases(typename V2<R>::T* __restrict__ amps, TileDesc td, const Phase* __restrict__ phases, int nphases,
               const PhaseOp<R>* __restrict__ ops, uint64_t gbase, uint64_t ntiles, FuseArgs fa)
{
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    T* s = reinterpret_cast<T*>(smem);
    uint32_t* cw = reinterpret_cast<uint32_t*>(smem + (sizeof(T) << kT));
    __shared__ uint64_t rowoff[1 << (kT - kPhaseLowBits)];
    const int l = td.l;  // 5 (rows of 32 amplitudes) or 8 (rows = codec block pairs)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nrows = 1u << (kT - l), rmask = (1u << l) - 1u;
    for (uint32_t rw = threadIdx.x; rw < nrows; rw += kThreads) {
        uint64_t off = 0;
        for (int i = 0; i < kT - l; i++)
            if ((rw >> i) & 1u) off |= 1ull << td.hpos[i];
        rowoff[rw] = off;
    }
    const uint64_t cmask = (1ull << fa.c) - 1;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = 0;
        for (int i = 0; i < td.nout; i++)
            if ((tile >> i) & 1ull) base |= 1ull << td.opos[i];
        __syncthreads();
        if (fa.decode) {
            // compressed streams -> shared: one warp per 256-amplitude block pair (row)
            for (uint32_t rw = wid; rw < nrows; rw += kThreads / 32) {
                const uint64_t li = base + rowoff[rw];
                const uint32_t r = (uint32_t)(li >> fa.c);
                const uint32_t bp = (uint32_t)((li & cmask) >> 8);
                R x[2][8];
                if (!codec::decode_pair<R>(fa.in + (size_t)r * fa.in_stride, fa.gin.bytes[r], fa.in_stride, fa.c,
                                           fa.dtype, bp, reinterpret_cast<uint32_t(*)[264]>(cw + wid * kCodecWords),
                                           (R)fa.scale, x, lane)) {
                    if (lane == 0) atomicOr(fa.err, kErrCorrupt);
#pragma unroll
                    for (int m = 0; m < 8; m++) x[0][m] = x[1][m] = (R)0;
                }
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    T v;
                    v.x = x[0][m];
                    v.y = x[1][m];
                    s[swz(rw * 256u + 8u * lane + m)] = v;
                }
            }
        } else {
            // HBM -> shared: 2 amplitudes (16 bytes for complex64) per access along rows
            for (uint32_t e = threadIdx.x; e < kN / 2; e += kThreads) {
                const uint32_t i = 2 * e;
                const T* g = amps + base + rowoff[i >> l] + (i & rmask);
                T x0, x1;
                if (sizeof(R) == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(g);
                    x0.x = v.x; x0.y = v.y; x1.x = v.z; x1.y = v.w;
                } else {
                    x0 = g[0];
                    x1 = g[1];
                }
                s[swz(i)] = x0;
                s[swz(i + 1)] = x1;
            }
        }
        __syncthreads();
        for (int ph = 0; ph < nphases; ph++) {
            const Phase P = phases[ph];
            uint32_t tb = 0;
#pragma unroll
            for (int j = 0; j < kT - kPhaseRegBits; j++) tb |= ((threadIdx.x >> j) & 1u) << P.tpos[j];
            uint32_t roff[kRegs];
#pragma unroll
            for (int m = 0; m < kRegs; m++) {
                uint32_t o = 0;
#pragma unroll
                for (int j = 0; j < kPhaseRegBits; j++)
                    if ((m >> j) & 1) o |= 1u << P.rpos[j];
                roff[m] = o;
            }
            T a[kRegs];
#pragma unroll
            for (int m = 0; m < kRegs; m++) a[m] = s[swz(tb | roff[m])];
            for (int oi = P.op_begin; oi < P.op_begin + P.op_count; oi++) {
                const PhaseOp<R>& op = ops[oi];
                if ((base & op.cmask_local) != op.cmask_local || (gbase & op.cmask_global) != op.cmask_global) continue;
                if ((tb & op.cmask_tile) != op.cmask_tile) continue;
                const uint32_t rm = op.cmask_reg;
                if (op.type == POP_DIAG) apply_diag<T, R>(op, a, tb, base, gbase, rm);
                else if (op.type == POP_DENSE2) apply_d2<T, R>(op.r0, op.r1, a, op.m, rm);
                else apply_d1<T, R>(op.type, op.r0, a, op.m, rm);
            }
#pragma unroll
            for (int m = 0; m < kRegs; m++) s[swz(tb | roff[m])] = a[m];
            __syncthreads();
        }
        if (fa.encode) {
            // shared -> codec: one warp per block pair; packed words go to the staging slots
            const CodecLayout CL = codec_layout(fa.c);
            for (uint32_t rw = wid; rw < nrows; rw += kThreads / 32) {
                const uint64_t li = base + rowoff[rw];
                const uint32_t r = (uint32_t)(li >> fa.c);
                const uint32_t bp = (uint32_t)((li & cmask) >> 8);
                R x[2][8];
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const T v = s[swz(rw * 256u + 8u * lane + m)];
                    x[0][m] = v.x;
                    x[1][m] = v.y;
                }
                codec::encode_pair<R>(x, fa.c, fa.k, bp, fa.out + (size_t)r * fa.out_stride,
                                      fa.sparse + (uint64_t)r * CL.nb * 256ull, fa.blocksq + (uint64_t)r * CL.bpc + bp,
                                      reinterpret_cast<uint32_t(*)[260]>(cw + wid * kCodecWords), fa.err, lane);
            }
        } else {
            for (uint32_t e = threadIdx.x; e < kN / 2; e += kThreads) {
                const uint32_t i = 2 * e;
                T* g = amps + base + rowoff[i >> l] + (i & rmask);
                const T x0 = s[swz(i)], x1 = s[swz(i + 1)];
                if (sizeof(R) == 4) {
                    *reinterpret_cast<float4*>(g) = make_float4((float)x0.x, (float)x0.y, (float)x1.x, (float)x1.y);
                } else {
                    g[0] = x0;
                    g[1] = x1;
                }
            }
        }
    }
}

}  // namespace

template <typename R>
cudaError_t launch_apply_phases(void* amps, const TileDesc& td, const Phase* phases, int nphases,
                                const PhaseOp<R>* ops, uint64_t gbase, const FuseArgs& fa, cudaStream_t st)
{
    static bool attr_set = false;
    const size_t smem = (sizeof(typename V2<R>::T) << kT) + sizeof(uint32_t) * kCodecWords * (kThreads / 32);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_apply_phases<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (td.l != 5 && td.l != 8) return cudaErrorInvalidValue;
    if ((fa.decode || fa.encode) && td.l != 8) return cudaErrorInvalidValue;
    const uint64_t ntiles = 1ull << (td.L - kT);
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, 152ull * 32);
    k_apply_phases<R><<<grid, kThreads, smem, st>>>(static_cast<typename V2<R>::T*>(amps), td, phases, nphases, ops,
                                                    gbase, ntiles, fa);
    return cudaGetLastError();
}

template cudaError_t launch_apply_phases<float>(void*, const TileDesc&, const Phase*, int, const PhaseOp<float>*,
                                                uint64_t, const FuseArgs&, cudaStream_t);
template cudaError_t launch_apply_phases<double>(void*, const TileDesc&, const Phase*, int, const PhaseOp<double>*,
                                                 uint64_t, const FuseArgs&, cudaStream_t);

}  // namespace sv
