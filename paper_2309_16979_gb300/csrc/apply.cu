// apply.cu -- gate application on staged chunk groups (MEMQSim Sec. 2,
// "Online stage" step (3): the GPU kernel that updates the state vector
// amplitudes), and the adjoint reverse sweep for gradients.
//
// A sub-pass loads one tile of 2^t amplitudes per CTA into shared memory --
// the amplitudes that vary over the tile's t local qubits with every other
// local bit fixed -- applies every gate of the sub-pass whose mixing qubits
// are tile qubits, and writes the tile back: one HBM read and one write per
// amplitude for the whole gate list. Tile rows are 2^l contiguous amplitudes
// (l >= 1) loaded with 16-byte vectors. Controls and diagonal factors on qubits
// outside the tile are evaluated once per CTA from the tile's fixed bits and
// the group's fixed high bits.
#include <algorithm>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kThreads = 256;

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

template <typename T, typename R>
__device__ __forceinline__ T cmul(R ar, R ai, T b)
{
    T o;
    o.x = ar * b.x - ai * b.y;
    o.y = ar * b.y + ai * b.x;
    return o;
}
template <typename T, typename R>
__device__ __forceinline__ T cmad(R ar, R ai, T b, T acc)
{
    acc.x += ar * b.x - ai * b.y;
    acc.y += ar * b.y + ai * b.x;
    return acc;
}

__device__ __forceinline__ uint64_t deposit_tile(uint64_t tile, const TileDesc& td)
{
    uint64_t base = 0;
    for (int i = 0; i < td.nout; i++)
        if ((tile >> i) & 1ull) base |= 1ull << td.opos[i];
    return base;
}

template <typename T>
__device__ __forceinline__ void load_tile(T* s, const T* __restrict__ g, uint64_t base, const uint64_t* rowoff,
                                          int t, int l);
template <>
__device__ __forceinline__ void load_tile<float2>(float2* s, const float2* __restrict__ g, uint64_t base,
                                                  const uint64_t* rowoff, int t, int l)
{
    const uint32_t n2 = 1u << (t - 1), rmask = (1u << l) - 1u;
    float4* s4 = reinterpret_cast<float4*>(s);
    for (uint32_t e = threadIdx.x; e < n2; e += kThreads) {
        const uint32_t i = 2 * e;
        const uint64_t gi = base + rowoff[i >> l] + (i & rmask);
        s4[e] = *reinterpret_cast<const float4*>(g + gi);
    }
}
template <>
__device__ __forceinline__ void load_tile<double2>(double2* s, const double2* __restrict__ g, uint64_t base,
                                                   const uint64_t* rowoff, int t, int l)
{
    const uint32_t n = 1u << t, rmask = (1u << l) - 1u;
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) s[i] = g[base + rowoff[i >> l] + (i & rmask)];
}
template <typename T>
__device__ __forceinline__ void store_tile(const T* s, T* __restrict__ g, uint64_t base, const uint64_t* rowoff,
                                           int t, int l);
template <>
__device__ __forceinline__ void store_tile<float2>(const float2* s, float2* __restrict__ g, uint64_t base,
                                                   const uint64_t* rowoff, int t, int l)
{
    const uint32_t n2 = 1u << (t - 1), rmask = (1u << l) - 1u;
    const float4* s4 = reinterpret_cast<const float4*>(s);
    for (uint32_t e = threadIdx.x; e < n2; e += kThreads) {
        const uint32_t i = 2 * e;
        *reinterpret_cast<float4*>(g + base + rowoff[i >> l] + (i & rmask)) = s4[e];
    }
}
template <>
__device__ __forceinline__ void store_tile<double2>(const double2* s, double2* __restrict__ g, uint64_t base,
                                                    const uint64_t* rowoff, int t, int l)
{
    const uint32_t n = 1u << t, rmask = (1u << l) - 1u;
    for (uint32_t i = threadIdx.x; i < n; i += kThreads) g[base + rowoff[i >> l] + (i & rmask)] = s[i];
}

__device__ __forceinline__ uint32_t src_bit(int32_t src, uint64_t base, uint64_t gbase, uint32_t& tile_pos)
{
    // returns the constant bit for non-tile sources; sets tile_pos (or 32 = none) for tile sources
    tile_pos = 32;
    if (src < 0) return 0;
    if (src < SRC_LOCAL) { tile_pos = (uint32_t)(src - SRC_TILE); return 0; }
    if (src < SRC_GLOBAL) return (uint32_t)((base >> (src - SRC_LOCAL)) & 1ull);
    return (uint32_t)((gbase >> (src - SRC_GLOBAL)) & 1ull);
}

// apply one op to a shared-memory tile; every thread of the CTA calls this
template <typename R>
__device__ __forceinline__ void apply_op(typename V2<R>::T* s, const DevOp<R>& op, int t, uint64_t base,
                                         uint64_t gbase)
{
    using T = typename V2<R>::T;
    const uint32_t ct = op.cmask_tile;
    if (op.type == OP_DENSE1) {
        const int p = op.t0;
        const uint32_t pb = 1u << p, half = 1u << (t - 1);
        const R m0 = op.m[0], m1 = op.m[1], m2 = op.m[2], m3 = op.m[3];
        const R m4 = op.m[4], m5 = op.m[5], m6 = op.m[6], m7 = op.m[7];
        for (uint32_t j = threadIdx.x; j < half; j += kThreads) {
            const uint32_t i0 = ((j >> p) << (p + 1)) | (j & (pb - 1u)), i1 = i0 | pb;
            if ((i0 & ct) != ct) continue;
            const T a = s[i0], b = s[i1];
            T o0 = cmul<T, R>(m0, m1, a);
            o0 = cmad<T, R>(m2, m3, b, o0);
            T o1 = cmul<T, R>(m4, m5, a);
            o1 = cmad<T, R>(m6, m7, b, o1);
            s[i0] = o0;
            s[i1] = o1;
        }
    } else if (op.type == OP_DENSE2) {
        const int p0 = op.t0, p1 = op.t1;
        const int lo = min(p0, p1), hi = max(p0, p1);
        const uint32_t quarter = 1u << (t - 2);
        for (uint32_t j = threadIdx.x; j < quarter; j += kThreads) {
            uint32_t i = ((j >> lo) << (lo + 1)) | (j & ((1u << lo) - 1u));
            i = ((i >> hi) << (hi + 1)) | (i & ((1u << hi) - 1u));
            if ((i & ct) != ct) continue;
            uint32_t idx[4];
            T v[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                idx[a] = i | ((a & 1) ? (1u << p0) : 0u) | ((a & 2) ? (1u << p1) : 0u);
                v[a] = s[idx[a]];
            }
#pragma unroll
            for (int r = 0; r < 4; r++) {
                T acc;
                acc.x = (R)0;
                acc.y = (R)0;
#pragma unroll
                for (int a = 0; a < 4; a++) acc = cmad<T, R>(op.m[2 * (4 * r + a)], op.m[2 * (4 * r + a) + 1], v[a], acc);
                s[idx[r]] = acc;
            }
        }
    } else {  // OP_DIAG
        uint32_t tp0, tp1;
        const uint32_t cb = src_bit(op.d0, base, gbase, tp0) | (src_bit(op.d1, base, gbase, tp1) << 1);
        const R e0r = op.m[0], e0i = op.m[1], e1r = op.m[2], e1i = op.m[3];
        const R e2r = op.m[4], e2i = op.m[5], e3r = op.m[6], e3i = op.m[7];
        const uint32_t n = 1u << t;
        for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
            if ((i & ct) != ct) continue;
            uint32_t v = cb;
            if (tp0 < 32) v |= (i >> tp0) & 1u;
            if (tp1 < 32) v |= ((i >> tp1) & 1u) << 1;
            const R er = v == 0 ? e0r : v == 1 ? e1r : v == 2 ? e2r : e3r;
            const R ei = v == 0 ? e0i : v == 1 ? e1i : v == 2 ? e2i : e3i;
            s[i] = cmul<T, R>(er, ei, s[i]);
        }
    }
}

__device__ __forceinline__ bool cta_active(uint64_t cl, uint64_t cg, uint64_t base, uint64_t gbase)
{
    return (base & cl) == cl && (gbase & cg) == cg;
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_apply(typename V2<R>::T* __restrict__ amps, TileDesc td, const DevOp<R>* __restrict__ ops, int nops,
        uint64_t gbase, uint64_t ntiles)
{
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = td.t, l = td.l;
    T* s = reinterpret_cast<T*>(smem);
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(smem + (sizeof(T) << t));
    const uint32_t nrows = 1u << (t - l);
    for (uint32_t rw = threadIdx.x; rw < nrows; rw += kThreads) {
        uint64_t off = 0;
        for (int i = 0; i < t - l; i++)
            if ((rw >> i) & 1u) off |= 1ull << td.hpos[i];
        rowoff[rw] = off;
    }
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = deposit_tile(tile, td);
        __syncthreads();
        load_tile<T>(s, amps, base, rowoff, t, l);
        __syncthreads();
        for (int oi = 0; oi < nops; oi++) {
            const DevOp<R>& op = ops[oi];
            if (!cta_active(op.cmask_local, op.cmask_global, base, gbase)) continue;
            apply_op<R>(s, op, t, base, gbase);
            __syncthreads();
        }
        store_tile<T>(s, amps, base, rowoff, t, l);
    }
}

// Adjoint sweep over one sub-pass: for each op (already reversed and daggered
// on the host), if it carries a gradient slot, accumulate
// Im <lambda| G |psi> over the tile (G = X, Y or Z on the op's target) into
// gpart[slot * ntiles + tile] in FP64; then apply the op to psi and lambda.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_adjoint(typename V2<R>::T* __restrict__ psi, typename V2<R>::T* __restrict__ lam, TileDesc td,
          const DevOp<R>* __restrict__ ops, int nops, uint64_t gbase, uint64_t ntiles, double* __restrict__ gpart,
          uint64_t tile0, uint64_t tile_stride)
{
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[kThreads / 32];
    const int t = td.t, l = td.l;
    T* sp = reinterpret_cast<T*>(smem);
    T* sl = sp + (1u << t);
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(smem + 2 * (sizeof(T) << t));
    const uint32_t nrows = 1u << (t - l);
    for (uint32_t rw = threadIdx.x; rw < nrows; rw += kThreads) {
        uint64_t off = 0;
        for (int i = 0; i < t - l; i++)
            if ((rw >> i) & 1u) off |= 1ull << td.hpos[i];
        rowoff[rw] = off;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = deposit_tile(tile, td);
        __syncthreads();
        load_tile<T>(sp, psi, base, rowoff, t, l);
        load_tile<T>(sl, lam, base, rowoff, t, l);
        __syncthreads();
        for (int oi = 0; oi < nops; oi++) {
            const DevOp<R>& op = ops[oi];
            if (op.grad_slot >= 0) {
                const int p = op.t0;
                const uint32_t pb = 1u << p, half = 1u << (t - 1);
                R acc = (R)0;  // imaginary part of the sum, thread-local over a few pairs
                for (uint32_t j = threadIdx.x; j < half; j += kThreads) {
                    const uint32_t i0 = ((j >> p) << (p + 1)) | (j & (pb - 1u)), i1 = i0 | pb;
                    const T p0 = sp[i0], p1 = sp[i1], l0 = sl[i0], l1 = sl[i1];
                    // Im(conj(a) b) = a.x b.y - a.y b.x
                    if (op.gen == 1) {        // X: conj(l0) p1 + conj(l1) p0
                        acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
                    } else if (op.gen == 2) { // Y: conj(l0)(-i p1) + conj(l1)(i p0); Im(conj(a)(i b)) = Re(conj(a) b)
                        acc += -(l0.x * p1.x + l0.y * p1.y) + (l1.x * p0.x + l1.y * p0.y);
                    } else {                  // Z: conj(l0) p0 - conj(l1) p1
                        acc += (l0.x * p0.y - l0.y * p0.x) - (l1.x * p1.y - l1.y * p1.x);
                    }
                }
                double d = (double)acc;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) d += __shfl_down_sync(FULL, d, o);
                if (lane == 0) red[wid] = d;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double sum = 0;
                    for (int w = 0; w < kThreads / 32; w++) sum += red[w];
                    gpart[(uint64_t)op.grad_slot * tile_stride + tile0 + tile] = sum;
                }
                // red[] is rewritten only after the next __syncthreads below
            }
            if (cta_active(op.cmask_local, op.cmask_global, base, gbase)) {
                apply_op<R>(sp, op, t, base, gbase);
                apply_op<R>(sl, op, t, base, gbase);
            }
            __syncthreads();
        }
        store_tile<T>(sp, psi, base, rowoff, t, l);
        store_tile<T>(sl, lam, base, rowoff, t, l);
    }
}

template <typename R>
size_t apply_smem(int t, int l, int tiles)
{
    return (size_t)tiles * (sizeof(typename V2<R>::T) << t) + (sizeof(uint64_t) << (t - l));
}

unsigned grid_for(uint64_t ntiles)
{
    return (unsigned)std::min<uint64_t>(ntiles, 152ull * 64);
}

}  // namespace

template <typename R>
cudaError_t launch_apply(void* amps, const TileDesc& td, const DevOp<R>* ops, int nops, uint64_t gbase,
                         cudaStream_t st)
{
    static bool attr_set = false;
    const size_t smem = apply_smem<R>(td.t, td.l, 1);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_apply<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)apply_smem<R>(kMaxTileQubits, 1, 1));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint64_t ntiles = 1ull << (td.L - td.t);
    k_apply<R><<<grid_for(ntiles), kThreads, smem, st>>>(static_cast<typename V2<R>::T*>(amps), td, ops, nops,
                                                         gbase, ntiles);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint(void* psi, void* lam, const TileDesc& td, const DevOp<R>* ops, int nops,
                           uint64_t gbase, double* gpart, uint64_t tile_stride, cudaStream_t st)
{
    static bool attr_set = false;
    const size_t smem = apply_smem<R>(td.t, td.l, 2);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)apply_smem<R>(kMaxTileQubits - 1, 1, 2));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint64_t ntiles = 1ull << (td.L - td.t);
    k_adjoint<R><<<grid_for(ntiles), kThreads, smem, st>>>(static_cast<typename V2<R>::T*>(psi),
                                                           static_cast<typename V2<R>::T*>(lam), td, ops, nops,
                                                           gbase, ntiles, gpart, 0, tile_stride);
    return cudaGetLastError();
}

template cudaError_t launch_apply<float>(void*, const TileDesc&, const DevOp<float>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_apply<double>(void*, const TileDesc&, const DevOp<double>*, int, uint64_t, cudaStream_t);
template cudaError_t launch_adjoint<float>(void*, void*, const TileDesc&, const DevOp<float>*, int, uint64_t,
                                           double*, uint64_t, cudaStream_t);
template cudaError_t launch_adjoint<double>(void*, void*, const TileDesc&, const DevOp<double>*, int, uint64_t,
                                            double*, uint64_t, cudaStream_t);

}  // namespace sv
