// apply_phase.cu -- register-phase gate application on 2^12-amplitude tiles
// (MEMQSim Sec. 2, "Online stage" step (3): the kernel that updates the
// amplitudes of the staged chunks).
//
// One CTA of 256 threads owns one tile of 4096 amplitudes at a time. The tile
// is read from HBM once (16-byte vectors along contiguous rows) into shared
// memory and written back once -- or, when the codec is fused, decoded from /
// encoded to the compressed chunk streams. In between, the sub-pass's gates
// run in phases: in a phase every thread holds the 16 amplitudes that vary
// over four tile qubits (the phase's register qubits) and applies, in
// registers, every gate whose mixing qubits are among them; the other eight
// tile bits are the thread's index. Controls and diagonal bits on
// non-register tile bits are per-thread constants, those outside the tile
// per-CTA constants.
//
// Per-gate cost is kept to the arithmetic: the sub-pass's phases and ops are
// staged in shared memory once per CTA; each op is one record whose dense
// `code` selects, through one jump table, code specialised at compile time
// for its form (real 2x2, RX-like 2x2, general 2x2, diagonals),
// target register bit and whether it has register controls (a host-computed
// 16-bit mask of the register indices that take part).
//
// Shared memory holds the tile XOR-swizzled (tile_dev.cuh); a phase's element
// address is swz(thread bits) ^ sroff[m], the sixteen register offsets
// pre-swizzled on the host.
#include <algorithm>

#include "sv_internal.h"
#include "tile_dev.cuh"

namespace sv {
namespace {

using tile::kThreads;
using tile::kT;
using tile::kN;
using tile::kCodecWords;
using tile::swz;
using tile::V2;
constexpr int kRegs = 1 << kPhaseRegBits;
constexpr int kMaxStagedOps = 256;      // ops staged in shared memory per launch
constexpr int kMaxStagedPhases = 64;    // phases staged in shared memory per launch

// Phase and op tables of the current pass in constant memory: read with a
// warp-uniform index they are uniform values, so the per-op dispatch is a
// uniform branch. Passes whose tables do not fit use the shared-memory path.
__constant__ Phase c_phases[kConstPhases];
__constant__ PhaseOp<float> c_ops_f[kConstOpsF];
__constant__ PhaseOp<double> c_ops_d[kConstOpsD];

template <typename R> __device__ __forceinline__ const PhaseOp<R>& cop(int i);
template <> __device__ __forceinline__ const PhaseOp<float>& cop<float>(int i) { return c_ops_f[i]; }
template <> __device__ __forceinline__ const PhaseOp<double>& cop<double>(int i) { return c_ops_d[i]; }

__device__ __forceinline__ uint32_t const_bit(uint8_t s, uint32_t tb, uint64_t base, uint64_t gbase)
{
    if (s == kSrcNone) return 0;
    if (s < 0x40) return (tb >> s) & 1u;
    if (s < 0x80) return (uint32_t)((base >> (s - 0x40)) & 1ull);
    return (uint32_t)((gbase >> (s - 0x80)) & 1ull);
}

// ------------------------------------------------------ 2x2 forms on bit B
template <int B, bool C, typename T, typename R>
__device__ __forceinline__ void f_generic(T (&a)[kRegs], const R* m, uint32_t am)
{
    const R m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3], m4 = m[4], m5 = m[5], m6 = m[6], m7 = m[7];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if (C && !((am >> i) & 1u)) continue;
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

template <int B, bool C, typename T, typename R>
__device__ __forceinline__ void f_real(T (&a)[kRegs], const R* m, uint32_t am)
{
    const R m0 = m[0], m2 = m[2], m4 = m[4], m6 = m[6];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if (C && !((am >> i) & 1u)) continue;
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
template <int B, bool C, typename T, typename R>
__device__ __forceinline__ void f_rx(T (&a)[kRegs], const R* m, uint32_t am)
{
    const R p = m[0], q = m[3], r = m[5], s = m[6];
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & (1 << B)) continue;
        if (C && !((am >> i) & 1u)) continue;
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

template <typename T, typename R>
__device__ __forceinline__ T cmul(R er, R ei, T x)
{
    T o;
    o.x = er * x.x - ei * x.y;
    o.y = er * x.y + ei * x.x;
    return o;
}

// diagonal whose entry index has one register bit B; the other index bit is
// constant per thread and selects the pair of factors
template <int B, bool C, typename T, typename R>
__device__ __forceinline__ void f_diag1(T (&a)[kRegs], const PhaseOp<R>& op, uint32_t tb, uint64_t base,
                                        uint64_t gbase)
{
    const uint32_t cb = const_bit(op.csrc, tb, base, gbase);
    const uint32_t lo = op.rsel ? cb : (cb << 1), hi = op.rsel ? (cb | 2u) : ((cb << 1) | 1u);
    const R lr = op.m[2 * lo], li = op.m[2 * lo + 1], hr = op.m[2 * hi], hv = op.m[2 * hi + 1];
    const uint32_t am = op.amask;
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (C && !((am >> i) & 1u)) continue;
        a[i] = (i & (1 << B)) ? cmul<T, R>(hr, hv, a[i]) : cmul<T, R>(lr, li, a[i]);
    }
}

template <int B0, int B1, bool C, typename T, typename R>
__device__ __forceinline__ void f_diag2(T (&a)[kRegs], const R* m, uint32_t am)
{
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (C && !((am >> i) & 1u)) continue;
        const int v = ((i >> B0) & 1) | (((i >> B1) & 1) << 1);
        a[i] = cmul<T, R>(m[2 * v], m[2 * v + 1], a[i]);
    }
}

template <bool C, typename T, typename R>
__device__ __forceinline__ void f_diagt(T (&a)[kRegs], const PhaseOp<R>& op, uint32_t tb, uint64_t base,
                                        uint64_t gbase)
{
    const uint32_t v = const_bit(op.csrc, tb, base, gbase) | (const_bit(op.csrc1, tb, base, gbase) << 1);
    const R er = op.m[2 * v], ei = op.m[2 * v + 1];
    const uint32_t am = op.amask;
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (C && !((am >> i) & 1u)) continue;
        a[i] = cmul<T, R>(er, ei, a[i]);
    }
}

template <int B0, int B1, typename T, typename R>
__device__ __forceinline__ void f_dense2(T (&a)[kRegs], const R* m, uint32_t am)
{
#pragma unroll
    for (int i = 0; i < kRegs; i++) {
        if (i & ((1 << B0) | (1 << B1))) continue;
        if (!((am >> i) & 1u)) continue;
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

// 4x4 ops are rare (two-target custom gates): they run out of line on the
// thread's own 16 shared-memory slots, so the register array is never
// addressed and stays in registers on the common path.
template <typename T, typename R>
__device__ __noinline__ void apply_dense2_smem(uint32_t bits, T* s, const uint16_t* sroff, uint32_t stb, const R* m,
                                               uint32_t am)
{
    T a[kRegs];
#pragma unroll
    for (int i = 0; i < kRegs; i++) a[i] = s[stb ^ sroff[i]];
    switch (bits) {  // b1 * 4 + b0
        case 0x4: f_dense2<0, 1, T, R>(a, m, am); break;
        case 0x8: f_dense2<0, 2, T, R>(a, m, am); break;
        case 0xc: f_dense2<0, 3, T, R>(a, m, am); break;
        case 0x1: f_dense2<1, 0, T, R>(a, m, am); break;
        case 0x9: f_dense2<1, 2, T, R>(a, m, am); break;
        case 0xd: f_dense2<1, 3, T, R>(a, m, am); break;
        case 0x2: f_dense2<2, 0, T, R>(a, m, am); break;
        case 0x6: f_dense2<2, 1, T, R>(a, m, am); break;
        case 0xe: f_dense2<2, 3, T, R>(a, m, am); break;
        case 0x3: f_dense2<3, 0, T, R>(a, m, am); break;
        case 0x7: f_dense2<3, 1, T, R>(a, m, am); break;
        case 0xb: f_dense2<3, 2, T, R>(a, m, am); break;
        default: break;
    }
#pragma unroll
    for (int i = 0; i < kRegs; i++) s[stb ^ sroff[i]] = a[i];
}

// Apply one staged op to the thread's 16 register amplitudes: one jump
// table over the dense op code (4x4 ops go through the thread's shared slots).
template <typename T, typename R>
__device__ __forceinline__ void apply_op(const PhaseOp<R>& op, T (&a)[kRegs], uint32_t tb, uint64_t base,
                                         uint64_t gbase, const R* __restrict__ dense2, T* s, const uint16_t* sroff,
                                         uint32_t stb)
{
    const uint32_t am = op.amask;
    const R* m = op.m;
#define SV_D1(K, FN)                                            \
    case K * 8 + 0: FN<0, false, T, R>(a, m, am); break;        \
    case K * 8 + 1: FN<1, false, T, R>(a, m, am); break;        \
    case K * 8 + 2: FN<2, false, T, R>(a, m, am); break;        \
    case K * 8 + 3: FN<3, false, T, R>(a, m, am); break;        \
    case K * 8 + 4: FN<0, true, T, R>(a, m, am); break;         \
    case K * 8 + 5: FN<1, true, T, R>(a, m, am); break;         \
    case K * 8 + 6: FN<2, true, T, R>(a, m, am); break;         \
    case K * 8 + 7: FN<3, true, T, R>(a, m, am); break;
#define SV_DG1(B, C) \
    case PK_DIAG1 * 8 + (C ? 4 : 0) + B: f_diag1<B, C, T, R>(a, op, tb, base, gbase); break;
#define SV_D2(B0, B1)                                                                        \
    case kCodeDiag2 + B1 * 4 + B0: f_diag2<B0, B1, false, T, R>(a, m, am); break;            \
    case kCodeDiag2 + 16 + B1 * 4 + B0: f_diag2<B0, B1, true, T, R>(a, m, am); break;
    switch (op.code) {
        SV_D1(PK_GENERIC, f_generic)
        SV_D1(PK_REAL, f_real)
        SV_D1(PK_RX, f_rx)
        SV_DG1(0, false) SV_DG1(1, false) SV_DG1(2, false) SV_DG1(3, false)
        SV_DG1(0, true) SV_DG1(1, true) SV_DG1(2, true) SV_DG1(3, true)
        SV_D2(0, 1) SV_D2(0, 2) SV_D2(0, 3) SV_D2(1, 0) SV_D2(1, 2) SV_D2(1, 3)
        SV_D2(2, 0) SV_D2(2, 1) SV_D2(2, 3) SV_D2(3, 0) SV_D2(3, 1) SV_D2(3, 2)
        case kCodeDiagT: f_diagt<false, T, R>(a, op, tb, base, gbase); break;
        case kCodeDiagT + 1: f_diagt<true, T, R>(a, op, tb, base, gbase); break;
        case kCodeDense2: {
#pragma unroll
            for (int i = 0; i < kRegs; i++) s[stb ^ sroff[i]] = a[i];
            apply_dense2_smem<T, R>(op.pad, s, sroff, stb, dense2 + 32ull * op.aux, am);
#pragma unroll
            for (int i = 0; i < kRegs; i++) a[i] = s[stb ^ sroff[i]];
            break;
        }
        default: break;
    }
#undef SV_D1
#undef SV_DG1
#undef SV_D2
}

template <typename R, bool CT>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 1)
k_apply_phases(typename V2<R>::T* __restrict__ amps, TileDesc td, const Phase* __restrict__ phases, int nphases,
               const PhaseOp<R>* __restrict__ ops, int op0, int nops, const CtaCtrl* __restrict__ ctl,
               const R* __restrict__ dense2, uint64_t gbase, uint64_t ntiles, FuseArgs fa, int ph_base)
{
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    T* s = reinterpret_cast<T*>(smem);
    const bool ph_staged = !CT && nphases <= kMaxStagedPhases;
    const bool op_staged = !CT && nops <= kMaxStagedOps;
    unsigned char* p = smem + (sizeof(T) << kT);
    Phase* sph = reinterpret_cast<Phase*>(p);
    p += ph_staged ? sizeof(Phase) * (size_t)nphases : 0;
    PhaseOp<R>* sops = reinterpret_cast<PhaseOp<R>*>(p);
    p += op_staged ? sizeof(PhaseOp<R>) * (size_t)nops : 0;
    uint32_t* cw = reinterpret_cast<uint32_t*>(p);
    __shared__ tile::Rows rt;
    tile::setup_rows(rt, td);
    if (ph_staged) {
        const uint4* src = reinterpret_cast<const uint4*>(phases);
        uint4* dst = reinterpret_cast<uint4*>(sph);
        const int nvec = (int)(sizeof(Phase) * (size_t)nphases / 16);
        for (int i = threadIdx.x; i < nvec; i += kThreads) dst[i] = src[i];
    }
    if (op_staged) {
        const uint4* src = reinterpret_cast<const uint4*>(ops + op0);
        uint4* dst = reinterpret_cast<uint4*>(sops);
        const int nvec = (int)(sizeof(PhaseOp<R>) * (size_t)nops / 16);
        for (int i = threadIdx.x; i < nvec; i += kThreads) dst[i] = src[i];
    }
    const Phase* phb = ph_staged ? sph : phases;
    const PhaseOp<R>* opb = op_staged ? sops : ops + op0;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        const uint64_t base = tile::tile_base(rt, td, tile);
        if (fa.decode) tile::load_tile<T, R, true>(s, amps, rt, td, base, fa, cw);
        else tile::load_tile<T, R, false>(s, amps, rt, td, base, fa, cw);
        __syncthreads();
        for (int ph = 0; ph < nphases; ph++) {
            const Phase& P = CT ? c_phases[ph_base + ph] : phb[ph];
            uint32_t tb = 0;
#pragma unroll
            for (int j = 0; j < kT - kPhaseRegBits; j++) tb |= ((threadIdx.x >> j) & 1u) << P.tpos[j];
            const uint32_t stb = swz(tb);
            T a[kRegs];
#pragma unroll
            for (int m = 0; m < kRegs; m++) a[m] = s[stb ^ P.sroff[m]];
            const int oe = P.op_begin - op0 + P.op_count;
            for (int oi = P.op_begin - op0; oi < oe; oi++) {
                const PhaseOp<R>& op = CT ? cop<R>(op0 + oi) : opb[oi];
                if (op.flags) {
                    const CtaCtrl cc = ctl[op.aux];
                    if ((base & cc.cl) != cc.cl || (gbase & cc.cg) != cc.cg) continue;
                }
                if ((tb & op.tmask) != op.tmask) continue;
                apply_op<T, R>(op, a, tb, base, gbase, dense2, s, P.sroff, stb);
            }
#pragma unroll
            for (int m = 0; m < kRegs; m++) s[stb ^ P.sroff[m]] = a[m];
            __syncthreads();
        }
        if (fa.encode) tile::store_tile<T, R, true>(s, amps, rt, td, base, fa, cw);
        else tile::store_tile<T, R, false>(s, amps, rt, td, base, fa, cw);
    }
}

}  // namespace

template <typename R> struct ConstOps;
template <> struct ConstOps<float> { static constexpr int cap = kConstOpsF; };
template <> struct ConstOps<double> { static constexpr int cap = kConstOpsD; };

template <typename R>
bool upload_const_tables(const Phase* phases, int nphases, const PhaseOp<R>* ops, int nops, cudaStream_t st)
{
    if (nphases > kConstPhases || nops > ConstOps<R>::cap) return false;
    if (nphases &&
        cudaMemcpyToSymbolAsync(c_phases, phases, sizeof(Phase) * nphases, 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return false;
    if (nops) {
        cudaError_t e = sizeof(R) == 4
                            ? cudaMemcpyToSymbolAsync(c_ops_f, ops, sizeof(PhaseOp<R>) * nops, 0, cudaMemcpyHostToDevice, st)
                            : cudaMemcpyToSymbolAsync(c_ops_d, ops, sizeof(PhaseOp<R>) * nops, 0, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return false;
    }
    return true;
}

template <typename R, bool CT>
static cudaError_t launch_impl(void* amps, const TileDesc& td, const Phase* phases, int nphases, const PhaseOp<R>* ops,
                               int op0, int nops, const CtaCtrl* ctl, const R* dense2, uint64_t gbase,
                               const FuseArgs& fa, cudaStream_t st, int ph_base)
{
    static bool attr_set = false;
    using T = typename V2<R>::T;
    const size_t codec_bytes = sizeof(uint32_t) * kCodecWords * (kThreads / 32);
    const size_t max_smem = (sizeof(T) << kT) + sizeof(Phase) * kMaxStagedPhases + sizeof(PhaseOp<R>) * kMaxStagedOps +
                            codec_bytes;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_apply_phases<R, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)max_smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const size_t smem = (sizeof(T) << kT) +
                        (!CT && nphases <= kMaxStagedPhases ? sizeof(Phase) * (size_t)nphases : 0) +
                        (!CT && nops <= kMaxStagedOps ? sizeof(PhaseOp<R>) * (size_t)nops : 0) +
                        ((fa.decode || fa.encode) ? codec_bytes : 0);
    const uint64_t ntiles = 1ull << (td.L - kT);
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, 152ull * 32);
    k_apply_phases<R, CT><<<grid, kThreads, smem, st>>>(static_cast<T*>(amps), td, phases, nphases, ops, op0, nops,
                                                        ctl, dense2, gbase, ntiles, fa, ph_base);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_apply_phases(void* amps, const TileDesc& td, const Phase* phases, int nphases,
                                const PhaseOp<R>* ops, int op0, int nops, const CtaCtrl* ctl, const R* dense2,
                                uint64_t gbase, const FuseArgs& fa, cudaStream_t st, int ph_base)
{
    if (td.l < tile::kMinLowBits || td.l > 8) return cudaErrorInvalidValue;
    if ((fa.decode || fa.encode) && td.l != 8) return cudaErrorInvalidValue;
    if (ph_base >= 0)
        return launch_impl<R, true>(amps, td, phases, nphases, ops, op0, nops, ctl, dense2, gbase, fa, st, ph_base);
    return launch_impl<R, false>(amps, td, phases, nphases, ops, op0, nops, ctl, dense2, gbase, fa, st, -1);
}

template bool upload_const_tables<float>(const Phase*, int, const PhaseOp<float>*, int, cudaStream_t);
template bool upload_const_tables<double>(const Phase*, int, const PhaseOp<double>*, int, cudaStream_t);
template cudaError_t launch_apply_phases<float>(void*, const TileDesc&, const Phase*, int, const PhaseOp<float>*, int,
                                                int, const CtaCtrl*, const float*, uint64_t, const FuseArgs&,
                                                cudaStream_t, int);
template cudaError_t launch_apply_phases<double>(void*, const TileDesc&, const Phase*, int, const PhaseOp<double>*,
                                                 int, int, const CtaCtrl*, const double*, uint64_t, const FuseArgs&,
                                                 cudaStream_t, int);

}  // namespace sv
