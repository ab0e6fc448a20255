// reduce.cu -- FP64 reductions over staged amplitudes: Pauli-sum expectation
// values, <a|b> dot products, the amplitude gather behind sv_amplitudes, and
// lambda = H psi for the adjoint gradient.
//
// Reductions are deterministic: each CTA covers a fixed index range, each
// thread first sums a few products in the amplitude precision, the per-thread
// sums are added in FP64 in a fixed tree, and per-CTA partials are summed in
// FP64 in index order by a final one-CTA-per-term kernel.
#include <algorithm>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kPerThread = 16;  // products summed in amplitude precision before FP64

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

__device__ __forceinline__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; w++) s += red[w];
    return s;
}

// partials[t * nblocks + block] = Re sum_{i in block range} conj(B[i ^ xl]) * phase_t(i) * A[i]
// phase_t(i) = i^ny * (-1)^(popcount(i & zl) + popcount(gbase & zg)).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pauli(const typename V2<R>::T* __restrict__ A, const typename V2<R>::T* __restrict__ B, uint64_t count,
        uint64_t gbase, const PauliDev* __restrict__ terms, int nterms, double* __restrict__ partials)
{
    __shared__ double red[kThreads / 32];
    const uint64_t per_block = (count + gridDim.x - 1) / gridDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * per_block;
    const uint64_t i1 = min(count, i0 + per_block);
    for (int tt = 0; tt < nterms; tt++) {
        const PauliDev P = terms[tt];
        const int gsign = __popcll(gbase & P.zg) & 1;
        double acc = 0;
        R sub = (R)0;
        int cnt = 0;
        for (uint64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
            const typename V2<R>::T a = A[i], b = B[i ^ P.xl];
            // Re(conj(b) * a) and Im(conj(b) * a)
            const R re = b.x * a.x + b.y * a.y;
            const R im = b.x * a.y - b.y * a.x;
            R v;
            switch (P.ny & 3) {  // multiply by i^ny, keep the real part
                case 0: v = re; break;
                case 1: v = -im; break;
                case 2: v = -re; break;
                default: v = im; break;
            }
            if ((__popcll(i & P.zl) + gsign) & 1) v = -v;
            sub += v;
            if (++cnt == kPerThread) {
                acc += (double)sub;
                sub = (R)0;
                cnt = 0;
            }
        }
        acc += (double)sub;
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) partials[(uint64_t)tt * gridDim.x + blockIdx.x] = s * P.coeff;
    }
}

// All terms in one sweep: partials[block] = sum_{i in block range}
// Re conj(psi_i) * sum_t coeff_t * phase_t(i) * psi[i ^ xl_t], i.e. the
// block's share of <psi|H|psi> over the buffer (phase_t as in k_pauli). The
// per-amplitude sum over terms runs in the amplitude precision, then FP64 as
// in k_pauli. Terms staged in shared memory.
//
// A thread holds a strip of 8 amplitudes, index i + 256 k (k = 0..7), and a
// CTA's strips start at multiples of 2048, so bits 8..10 of i are zero and a
// term's sign (-1)^popcount(j & z) is the sign of i (one popcount per strip)
// times a per-term table over k. For a term with an x mask, the amplitudes j
// and j ^ x contribute equal real parts (the term is Hermitian); when the
// lowest bit of x is one of the strip bits (8..10) or above, only the member
// of each pair with that bit clear is evaluated, with twice the coefficient
// (the choice is the same for the whole strip or the whole CTA, so warps do
// not diverge).
constexpr int kMaxEnergyTerms = 512;

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_energy(const typename V2<R>::T* __restrict__ psi, uint64_t count, uint64_t gbase, const PauliDev* __restrict__ terms,
         int nterms, double* __restrict__ partials)
{
    constexpr int kStrip = 8;
    constexpr uint64_t kSpan = (uint64_t)kThreads * kStrip;  // 2048 amplitudes: one strip of the CTA
    __shared__ double red[kThreads / 32];
    __shared__ uint64_t sx[kMaxEnergyTerms], sz[kMaxEnergyTerms];
    __shared__ R sre[kMaxEnergyTerms], sim[kMaxEnergyTerms];
    __shared__ uint32_t stab[kMaxEnergyTerms];
    for (int t = threadIdx.x; t < nterms; t += kThreads) {
        const PauliDev P = terms[t];
        sx[t] = P.xl;
        sz[t] = P.zl;
        // the global-bit sign folded into the coefficient; doubled where one
        // member of each pair is evaluated
        double cf = (__popcll(gbase & P.zg) & 1) ? -P.coeff : P.coeff;
        if (P.xl != 0 && (P.xl & 0xFFull) == 0) cf *= 2.0;
        // real part of i^ny-weighted conj(psi_j) psi_{j^x} as cr*re + ci*im
        // (re, im as below; the sign of z on x's bits folded in, as in k_pauli)
        const int ny = P.ny & 3;
        sre[t] = (R)(ny == 0 ? cf : ny == 2 ? -cf : 0.0);
        sim[t] = (R)(ny == 1 ? -cf : ny == 3 ? cf : 0.0);
        // bit k: parity of z on the strip bits of k
        uint32_t tab = 0;
        for (int k = 0; k < kStrip; k++) tab |= (uint32_t)(__popcll(((uint64_t)k << 8) & P.zl) & 1) << k;
        stab[t] = tab;
    }
    __syncthreads();
    const uint64_t per_block = ((count + gridDim.x - 1) / gridDim.x + kSpan - 1) / kSpan * kSpan;
    const uint64_t i0 = (uint64_t)blockIdx.x * per_block;
    const uint64_t i1 = min(count, i0 + per_block);
    using T = typename V2<R>::T;
    double acc = 0;
    for (uint64_t s0 = i0; s0 < i1; s0 += kSpan) {
        const uint64_t i = s0 + threadIdx.x;
        T a[kStrip];
        R e[kStrip], n2[kStrip];
#pragma unroll
        for (int k = 0; k < kStrip; k++) {
            const uint64_t j = i + (uint64_t)k * kThreads;
            a[k] = j < i1 ? psi[j] : T{(R)0, (R)0};
            e[k] = (R)0;
            n2[k] = a[k].x * a[k].x + a[k].y * a[k].y;
        }
        for (int t = 0; t < nterms; t++) {
            const uint64_t x = sx[t];
            const uint32_t sg = stab[t] ^ ((__popcll(i & sz[t]) & 1) ? 0xFFu : 0u);  // bit k: sign of j_k
            const R cr = sre[t];
            if (x == 0) {
                // a Z string (no Y without an X): |psi_j|^2 with its sign
#pragma unroll
                for (int k = 0; k < kStrip; k++) e[k] += (((sg >> k) & 1u) ? -cr : cr) * n2[k];
                continue;
            }
            const uint64_t xb = x & (~x + 1);  // lowest bit of x
            if (xb >= kSpan && (s0 & xb)) continue;  // the strip s0 ^ xb evaluates these pairs
            const R ci = sim[t];
#pragma unroll
            for (int k = 0; k < kStrip; k++) {
                const uint64_t kb = (uint64_t)k * kThreads;
                if (xb >= (uint64_t)kThreads && xb < kSpan && (kb & xb)) continue;  // counted at k ^ (xb >> 8)
                const uint64_t j = i + kb;
                const T b = j < i1 ? psi[j ^ x] : T{(R)0, (R)0};
                const R re = b.x * a[k].x + b.y * a[k].y;
                const R im = b.x * a[k].y - b.y * a[k].x;
                const R v = cr * re + ci * im;
                e[k] += ((sg >> k) & 1u) ? -v : v;
            }
        }
        R sub = (R)0;
#pragma unroll
        for (int k = 0; k < kStrip; k++) sub += e[k];
        acc += (double)sub;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Bulk (TMA) copies into shared memory completing on an mbarrier, and a
// bounded wait for them.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16; both addresses 16-byte aligned) from global to shared
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// true once the barrier's phase of this parity has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr uint32_t kWaitPolls = 1u << 22;

// The same sum as k_energy for terms whose x-masks lie in a tile's bits
// (local bits 0..7 and et.hp[0..3]): a CTA holds a tile of 4096 amplitudes
// (16 rows of 256 contiguous ones) in shared memory and every term's
// partner is read there, so the buffer is read once for all these terms
// instead of once more per term. Both members of a pair are evaluated (the
// coefficient is not doubled). Thread t holds tile positions t + 256k,
// k = 0..15; a tile position's local index is the tile base | t | the
// offsets of k's bits on hp. Tiles arrive as 16 bulk row copies on an
// mbarrier, double-buffered: the CTA's next tile is in flight while the
// current one is evaluated. Per tile, products in the amplitude precision;
// across tiles FP64; a fixed reduction tree. A wait that exceeds its limit
// sets kErrWait and ends the CTA's work.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_energy_tiles(const typename V2<R>::T* __restrict__ psi, uint64_t ntiles, uint64_t gbase, const EnergyTiles et,
               const PauliDev* __restrict__ terms, int nterms, double* __restrict__ partials, int* __restrict__ err)
{
    using T = typename V2<R>::T;
    constexpr uint32_t kTile = 1u << kEnergyTileBits;
    extern __shared__ __align__(128) unsigned char tile_smem[];  // two tiles of 4096 amplitudes
    T* const buf = reinterpret_cast<T*>(tile_smem);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int ok_s;
    __shared__ double red[kThreads / 32];
    __shared__ uint32_t sxt[kMaxEnergyTerms];   // x-mask on tile bits (bit 8 + i <-> hp[i])
    __shared__ uint64_t szl[kMaxEnergyTerms];   // z-mask on local bits
    __shared__ uint32_t srow[kMaxEnergyTerms];  // bit k: parity of z on k's row offset
    __shared__ R sre[kMaxEnergyTerms], sim[kMaxEnergyTerms];
    const uint32_t t = threadIdx.x;
    uint64_t rowoff[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        uint64_t o = 0;
        for (int i = 0; i < 4; i++)
            if ((k >> i) & 1) o |= 1ull << et.hp[i];
        rowoff[k] = o;
    }
    auto tile_base = [&](uint64_t tl) {
        uint64_t tb = 0;
        for (int i = 0; i < et.nout; i++)
            if ((tl >> i) & 1ull) tb |= 1ull << et.op[i];
        return tb;
    };
    // thread 0 issues a tile's 16 row copies into buffer b
    auto issue = [&](uint64_t tl, int b) {
        const uint64_t tb = tile_base(tl);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic reads of b came first
        mbar_expect_tx(&bar[b], kTile * (uint32_t)sizeof(T));
        for (int k = 0; k < 16; k++)
            bulk_load(buf + b * kTile + 256u * k, psi + tb + rowoff[k], 256u * (uint32_t)sizeof(T), &bar[b]);
    };
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int q = t; q < nterms; q += kThreads) {
        const PauliDev P = terms[q];
        uint32_t xt = (uint32_t)(P.xl & 0xFFull);
        for (int i = 0; i < 4; i++) xt |= (uint32_t)((P.xl >> et.hp[i]) & 1ull) << (8 + i);
        sxt[q] = xt;
        szl[q] = P.zl;
        const double cf = (__popcll(gbase & P.zg) & 1) ? -P.coeff : P.coeff;
        const int ny = P.ny & 3;
        sre[q] = (R)(ny == 0 ? cf : ny == 2 ? -cf : 0.0);
        sim[q] = (R)(ny == 1 ? -cf : ny == 3 ? cf : 0.0);
        uint32_t tab = 0;
        for (int k = 0; k < 16; k++) tab |= (uint32_t)(__popcll(rowoff[k] & P.zl) & 1) << k;
        uint32_t r = 0;  // z on the four row positions
        for (int i = 0; i < 4; i++) r |= (uint32_t)((P.zl >> et.hp[i]) & 1ull) << i;
        srow[q] = tab | (r << 16);
    }
    __syncthreads();
    bool pending[2] = {false, false};  // thread 0: a copy into the buffer not yet waited for
    if (t == 0 && blockIdx.x < ntiles) {
        issue(blockIdx.x, 0);
        pending[0] = true;
    }
    double acc = 0;
    uint32_t it = 0;
    for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, it++) {
        const int b = (int)(it & 1);
        const uint32_t parity = (it >> 1) & 1u;
        if (t == 0) {
            // the other buffer was last read in the previous iteration (a barrier ago)
            if (tl + gridDim.x < ntiles) {
                issue(tl + gridDim.x, b ^ 1);
                pending[b ^ 1] = true;
            }
            ok_s = mbar_wait(&bar[b], parity, kWaitPolls) ? 1 : 0;
            pending[b] = !ok_s;
        }
        __syncthreads();
        if (!ok_s) break;
        if (t != 0) mbar_wait(&bar[b], parity, kWaitPolls);  // complete already: this thread's acquire
        const T* const tile = buf + b * kTile;
        const uint64_t jt = tile_base(tl) | t;
        T a[16];
        R n2[16], e[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            a[k] = tile[t + 256u * k];
            n2[k] = a[k].x * a[k].x + a[k].y * a[k].y;
            e[k] = (R)0;
        }
        // diagonal terms: c (-1)^|j & z| with j = jt + row offset of k splits
        // into (-1)^|jt & z| and (-1)^|k & r| (r: z on the row positions), so
        // they sum per r into dc[r] and a 16-point Walsh-Hadamard transform
        // gives every row's coefficient at once
        R dc[16];
#pragma unroll
        for (int k = 0; k < 16; k++) dc[k] = (R)0;
        for (int q = 0; q < nterms; q++) {
            const uint32_t xt = sxt[q];
            const R cr = sre[q];
            if (xt == 0) {
                const R v = (__popcll(jt & szl[q]) & 1) ? -cr : cr;
                switch (srow[q] >> 16) {
#define SV_DC(i) case i: dc[i] += v; break;
                    SV_DC(0) SV_DC(1) SV_DC(2) SV_DC(3) SV_DC(4) SV_DC(5) SV_DC(6) SV_DC(7)
                    SV_DC(8) SV_DC(9) SV_DC(10) SV_DC(11) SV_DC(12) SV_DC(13) SV_DC(14) SV_DC(15)
#undef SV_DC
                }
                continue;
            }
            const uint32_t sg = (__popcll(jt & szl[q]) & 1) ? ~srow[q] : srow[q];  // bit k: sign of position k
            // Both members of a pair (position and partner) add the same
            // real value (P is Hermitian), so one member per pair adds it
            // twice: with a row bit flipped (pk != 0), the rows whose lowest
            // flipped row bit is clear; else the rows whose bit 0 equals the
            // thread's lowest flipped thread bit. Each thread takes 8 rows.
            const R c2r = cr + cr, c2i = sim[q] + sim[q];
            const uint32_t pt = t ^ (xt & 0xFFu), pk = xt >> 8;
#define SV_PAIR(k, own)                                                      \
    {                                                                        \
        const T bb = tile[pt + 256u * ((uint32_t)(k) ^ pk)];                 \
        const T aa = (own);                                                  \
        const R re = bb.x * aa.x + bb.y * aa.y;                              \
        const R im = bb.x * aa.y - bb.y * aa.x;                              \
        const R v = c2r * re + c2i * im;                                     \
        e[m] += ((sg >> (k)) & 1u) ? -v : v;                                 \
    }
#define SV_ROWPAIRS(PB)                                                      \
    _Pragma("unroll") for (int m = 0; m < 8; m++) {                          \
        const int k = ((m >> (PB)) << ((PB) + 1)) | (m & ((1 << (PB)) - 1)); \
        SV_PAIR(k, a[k])                                                     \
    }
            if (pk) {
                switch (__ffs(pk) - 1) {
                    case 0: SV_ROWPAIRS(0) break;
                    case 1: SV_ROWPAIRS(1) break;
                    case 2: SV_ROWPAIRS(2) break;
                    default: SV_ROWPAIRS(3) break;
                }
            } else {
                const uint32_t tb = (t >> (__ffs(xt & 0xFFu) - 1)) & 1u;
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    const uint32_t k = 2u * (uint32_t)m + tb;
                    SV_PAIR(k, tb ? a[2 * m + 1] : a[2 * m])
                }
            }
#undef SV_ROWPAIRS
#undef SV_PAIR
        }
#pragma unroll
        for (int h = 1; h < 16; h <<= 1)
#pragma unroll
            for (int i = 0; i < 16; i += 2 * h)
#pragma unroll
                for (int j = i; j < i + h; j++) {
                    const R a0 = dc[j], a1 = dc[j + h];
                    dc[j] = a0 + a1;
                    dc[j + h] = a0 - a1;
                }
        R sub = (R)0;
#pragma unroll
        for (int k = 0; k < 16; k++) sub += e[k] + dc[k] * n2[k];
        acc += (double)sub;
        __syncthreads();  // this buffer's reads are done before it is refilled
    }
    if (t == 0 && (pending[0] || pending[1])) {
        atomicOr(err, kErrWait);
        // copies still in flight must land before the CTA's shared memory goes away
        for (int b = 0; b < 2; b++)
            if (pending[b]) mbar_wait(&bar[b], ((it + (b != (int)(it & 1))) >> 1) & 1u, kWaitPolls);
    }
    const double sblk = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = sblk;
}

// out[t] += sum over blocks of partials[t * nblocks + b], one CTA per term, fixed order
__global__ void __launch_bounds__(kThreads)
k_sum_partials(const double* __restrict__ partials, int nblocks, double* __restrict__ out)
{
    __shared__ double red[kThreads / 32];
    const int tt = blockIdx.x;
    double acc = 0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) acc += partials[(uint64_t)tt * nblocks + b];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[tt] += s;
}

// <A|B> over a contiguous run of A: each CTA owns one contiguous index range,
// products in FP64, a fixed reduction tree (deterministic).
template <typename RA, typename RB>
__global__ void __launch_bounds__(kThreads)
k_inner(const typename V2<RA>::T* __restrict__ A, uint64_t count, uint64_t base,
        const typename V2<RB>::T* __restrict__ B, const IndexMap map, double* __restrict__ partials)
{
    __shared__ double red[kThreads / 32];
    const uint64_t per = (count + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = (uint64_t)blockIdx.x * per, hi = min(count, lo + per);
    double re = 0, im = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        const uint64_t pa = base + i;
        uint64_t pb = pa;
        if (!map.identity) {
            pb = 0;
            for (int j = 0; j < map.n; j++) pb |= ((pa >> j) & 1ull) << map.pos[j];
        }
        const typename V2<RA>::T a = A[i];
        const typename V2<RB>::T b = B[pb];
        const double ar = (double)a.x, ai = (double)a.y, br = (double)b.x, bi = (double)b.y;
        re += ar * br + ai * bi;
        im += ar * bi - ai * br;
    }
    const double sr = block_sum(re, red);
    const double si = block_sum(im, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sr;
        partials[gridDim.x + blockIdx.x] = si;
    }
}

template <typename R>
__global__ void k_gather(const typename V2<R>::T* __restrict__ amps, const uint64_t* __restrict__ local_idx,
                         const uint64_t* __restrict__ dest, uint64_t m, double* __restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const typename V2<R>::T a = amps[local_idx[i]];
        const uint64_t d = dest[i];
        out[2 * d] = (double)a.x;
        out[2 * d + 1] = (double)a.y;
    }
}

// lam[k] = sum_t coeff_t * phase_t(k ^ x_t) * psi[k ^ x_t]
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_hamiltonian(const typename V2<R>::T* __restrict__ psi, typename V2<R>::T* __restrict__ lam, uint64_t count,
              const PauliDev* __restrict__ terms, int nterms)
{
    using T = typename V2<R>::T;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (uint64_t)gridDim.x * blockDim.x) {
        R ar = (R)0, ai = (R)0;
        for (int tt = 0; tt < nterms; tt++) {
            const PauliDev& P = terms[tt];
            const uint64_t src = k ^ P.xl;
            const T v = psi[src];
            R vr = v.x, vi = v.y, tr;
            switch (P.ny & 3) {
                case 1: tr = vr; vr = -vi; vi = tr; break;   // * i
                case 2: vr = -vr; vi = -vi; break;
                case 3: tr = vr; vr = vi; vi = -tr; break;   // * -i
                default: break;
            }
            const R c = (__popcll(src & P.zl) & 1) ? (R)(-P.coeff) : (R)P.coeff;
            ar += c * vr;
            ai += c * vi;
        }
        T o;
        o.x = ar;
        o.y = ai;
        lam[k] = o;
    }
}

// One output chunk of lambda = H psi on compressed chunks: the source chunks
// k ^ xh of every distinct high x-mask are staged side by side (slot s at
// s << c); term t reads slot terms[t].pad, its low x-mask flips local bits,
// and the sign from its z-mask on the source chunk's high bits is already in
// its coefficient. The host orders the terms so that those reading the same
// source (slot and low x-mask) are consecutive: a run of them loads its
// source amplitudes once, sums its terms' coefficients c i^ny (-1)^|src & z|
// per output, and adds coefficient x source at the run's end.
// Each thread builds a strip of 8 outputs k = b + 256 m (b: the strip base
// plus the thread, bits 8..10 clear), so the 8 source reads of a run are in
// flight together while its coefficients are summed, and a term's sign
// (-1)^|(k ^ x) & z| splits into (-1)^|x & z|, taken when the term is
// staged, (-1)^|b & z|, once per thread, and a pattern over m from z's bits
// 8..10, staged with the term: most terms have none and add one coefficient
// to all 8 outputs.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_ham_chunk(const typename V2<R>::T* __restrict__ psi_slots, typename V2<R>::T* __restrict__ lam, int c,
            const PauliDev* __restrict__ terms, int nterms, int accumulate)
{
    using T = typename V2<R>::T;
    constexpr int kStrip = 8, kBatch = 256;
    static_assert(kThreads == 256 && kStrip == 8, "the sign pattern covers bits 8..10 of the output index");
    __shared__ uint64_t sxl[kBatch], szl[kBatch];
    __shared__ R sc[kBatch];            // c (-1)^|x & z| (-1)^[ny >= 2]
    __shared__ int32_t spad[kBatch];
    __shared__ uint32_t sfl[kBatch];    // sign pattern over m << 1 | ny odd
    const uint64_t count = 1ull << c;
    const uint64_t span = (uint64_t)kThreads * kStrip;
    for (uint64_t s0 = (uint64_t)blockIdx.x * span; s0 < count; s0 += (uint64_t)gridDim.x * span) {
        const uint64_t kb = s0 + threadIdx.x;
        R ar[kStrip], ai[kStrip];  // lambda
        R fr[kStrip], fi[kStrip];  // the current run's coefficient per output
        T v[kStrip];               // the current run's source amplitudes
#pragma unroll
        for (int m = 0; m < kStrip; m++) {
            const uint64_t k = kb + (uint64_t)m * kThreads;
            ar[m] = ai[m] = fr[m] = fi[m] = (R)0;
            v[m] = T{(R)0, (R)0};
            if (accumulate && k < count) {
                const T l = lam[k];
                ar[m] = l.x;
                ai[m] = l.y;
            }
        }
        int rpad = -1;      // the current run's slot (-1: none yet)
        uint64_t rxl = 0;   // and low x-mask
        bool rim = false;   // whether its coefficients have imaginary parts
        const bool whole = s0 + span <= count;
        for (int b0 = 0; b0 < nterms; b0 += kBatch) {
            const int nb = min(kBatch, nterms - b0);
            __syncthreads();
            for (int q = threadIdx.x; q < nb; q += kThreads) {
                const PauliDev& P = terms[b0 + q];
                R cf = (R)P.coeff;
                if (__popcll(P.xl & P.zl) & 1) cf = -cf;
                if (P.ny & 2) cf = -cf;
                uint32_t pat = 0;
#pragma unroll
                for (int m = 0; m < kStrip; m++)
                    pat |= (uint32_t)(__popcll(((uint64_t)m * kThreads) & P.zl) & 1) << m;
                sxl[q] = P.xl;
                szl[q] = P.zl;
                sc[q] = cf;
                spad[q] = P.pad;
                sfl[q] = (pat << 1) | (uint32_t)(P.ny & 1);
            }
            __syncthreads();
            for (int q = 0; q < nb; q++) {
                const uint64_t xl = sxl[q], zl = szl[q];
                const int pad = spad[q];
                const uint32_t fl = sfl[q], pat = fl >> 1;
                if (pad != rpad || xl != rxl) {
                    // a new source: finish the run before it, load this one
                    if (rpad >= 0 && rim) {
#pragma unroll
                        for (int m = 0; m < kStrip; m++) {
                            ar[m] += fr[m] * v[m].x - fi[m] * v[m].y;
                            ai[m] += fr[m] * v[m].y + fi[m] * v[m].x;
                            fr[m] = fi[m] = (R)0;
                        }
                    } else if (rpad >= 0) {
#pragma unroll
                        for (int m = 0; m < kStrip; m++) {
                            ar[m] += fr[m] * v[m].x;
                            ai[m] += fr[m] * v[m].y;
                            fr[m] = (R)0;
                        }
                    }
                    rpad = pad;
                    rxl = xl;
                    rim = false;
                    const T* const src_slot = psi_slots + ((uint64_t)pad << c);
                    if (whole && !(xl & (7ull << 8))) {
                        // k ^ x = (b ^ x) + 256 m: one base, constant offsets
                        const T* const sp = src_slot + (kb ^ xl);
#pragma unroll
                        for (int m = 0; m < kStrip; m++) v[m] = sp[m * kThreads];
                    } else {
#pragma unroll
                        for (int m = 0; m < kStrip; m++) {
                            const uint64_t k = kb + (uint64_t)m * kThreads;
                            v[m] = k < count ? src_slot[k ^ xl] : T{(R)0, (R)0};
                        }
                    }
                }
                const R w = (__popcll(kb & zl) & 1) ? -sc[q] : sc[q];
                if (pat == 0 && !(fl & 1)) {
#pragma unroll
                    for (int m = 0; m < kStrip; m++) fr[m] += w;
                } else if (pat == 0) {
                    rim = true;
#pragma unroll
                    for (int m = 0; m < kStrip; m++) fi[m] += w;
                } else if (!(fl & 1)) {
#pragma unroll
                    for (int m = 0; m < kStrip; m++) fr[m] += ((pat >> m) & 1) ? -w : w;
                } else {
                    rim = true;
#pragma unroll
                    for (int m = 0; m < kStrip; m++) fi[m] += ((pat >> m) & 1) ? -w : w;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < kStrip; m++) {
            const uint64_t k = kb + (uint64_t)m * kThreads;
            if (k < count) {
                T o;
                o.x = ar[m] + (fr[m] * v[m].x - fi[m] * v[m].y);
                o.y = ai[m] + (fr[m] * v[m].y + fi[m] * v[m].x);
                lam[k] = o;
            }
        }
    }
}

// partials[block] = Re sum conj(A[i]) B[i] over the block's range (FP64 accumulation)
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_dot(const typename V2<R>::T* __restrict__ A, const typename V2<R>::T* __restrict__ B, uint64_t count,
      double* __restrict__ partials)
{
    __shared__ double red[kThreads / 32];
    const uint64_t per_block = (count + gridDim.x - 1) / gridDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * per_block;
    const uint64_t i1 = min(count, i0 + per_block);
    double acc = 0;
    R sub = (R)0;
    int cnt = 0;
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
        const typename V2<R>::T a = A[i], b = B[i];
        sub += a.x * b.x + a.y * b.y;
        if (++cnt == kPerThread) {
            acc += (double)sub;
            sub = (R)0;
            cnt = 0;
        }
    }
    acc += (double)sub;
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

}  // namespace

int reduce_blocks_for(uint64_t count)
{
    const uint64_t want = (count + kThreads * 64 - 1) / (kThreads * 64);
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, 152ull * 8));
}

template <typename R>
cudaError_t launch_pauli_partials(const void* A, const void* B, int Lbits, uint64_t gbase, const PauliDev* terms,
                                  int nterms, double* partials, int nblocks, cudaStream_t st)
{
    using T = typename V2<R>::T;
    k_pauli<R><<<nblocks, kThreads, 0, st>>>(static_cast<const T*>(A), static_cast<const T*>(B), 1ull << Lbits,
                                            gbase, terms, nterms, partials);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_energy_partials(const void* psi, int Lbits, uint64_t gbase, const PauliDev* terms, int nterms,
                                   double* partials, int nblocks, cudaStream_t st)
{
    if (nterms > kMaxEnergyTerms) return cudaErrorInvalidValue;
    using T = typename V2<R>::T;
    k_energy<R><<<nblocks, kThreads, 0, st>>>(static_cast<const T*>(psi), 1ull << Lbits, gbase, terms, nterms,
                                             partials);
    return cudaGetLastError();
}

int max_energy_terms() { return kMaxEnergyTerms; }

cudaError_t launch_sum_partials(const double* partials, int nterms, int nblocks, double* out, cudaStream_t st)
{
    k_sum_partials<<<nterms, kThreads, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_energy_tiles(const void* psi, int Lbits, uint64_t gbase, const EnergyTiles& et,
                                const PauliDev* terms, int nterms, double* partials, int nblocks, int* err,
                                cudaStream_t st)
{
    if (Lbits < kEnergyTileBits || nterms > kMaxEnergyTerms) return cudaErrorInvalidValue;
    const uint64_t ntiles = 1ull << (Lbits - kEnergyTileBits);
    const int smem = (int)(2 * sizeof(typename V2<R>::T) << kEnergyTileBits);  // two tile buffers
    static thread_local int attr_device = -1;  // the attribute is per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_energy_tiles<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    k_energy_tiles<R><<<nblocks, kThreads, smem, st>>>(static_cast<const typename V2<R>::T*>(psi), ntiles, gbase, et,
                                                      terms, nterms, partials, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather(const void* amps, const uint64_t* local_idx, const uint64_t* dest, uint64_t m,
                          double* out, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<uint64_t>((m + 255) / 256, 152ull * 16);
    k_gather<R><<<blocks, 256, 0, st>>>(static_cast<const typename V2<R>::T*>(amps), local_idx, dest, m, out);
    return cudaGetLastError();
}

template <typename RA, typename RB>
cudaError_t launch_inner(const void* A, uint64_t count, uint64_t base, const void* B, const IndexMap& map,
                         double* partials, int nblocks, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    k_inner<RA, RB><<<nblocks, kThreads, 0, st>>>(static_cast<const typename V2<RA>::T*>(A), count, base,
                                                  static_cast<const typename V2<RB>::T*>(B), map, partials);
    return cudaGetLastError();
}

template cudaError_t launch_inner<float, float>(const void*, uint64_t, uint64_t, const void*, const IndexMap&,
                                                double*, int, cudaStream_t);
template cudaError_t launch_inner<float, double>(const void*, uint64_t, uint64_t, const void*, const IndexMap&,
                                                 double*, int, cudaStream_t);
template cudaError_t launch_inner<double, float>(const void*, uint64_t, uint64_t, const void*, const IndexMap&,
                                                 double*, int, cudaStream_t);
template cudaError_t launch_inner<double, double>(const void*, uint64_t, uint64_t, const void*, const IndexMap&,
                                                  double*, int, cudaStream_t);

template <typename R>
cudaError_t launch_hamiltonian(const void* psi, void* lam, int n, const PauliDev* terms, int nterms,
                               cudaStream_t st)
{
    using T = typename V2<R>::T;
    const uint64_t count = 1ull << n;
    const unsigned blocks = (unsigned)std::min<uint64_t>((count + kThreads - 1) / kThreads, 152ull * 32);
    k_hamiltonian<R><<<blocks, kThreads, 0, st>>>(static_cast<const T*>(psi), static_cast<T*>(lam), count, terms,
                                                 nterms);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ham_chunk(const void* psi_slots, void* lam, int c, const PauliDev* terms, int nterms,
                             bool accumulate, cudaStream_t st)
{
    using T = typename V2<R>::T;
    const uint64_t count = 1ull << c;
    const unsigned blocks = (unsigned)std::min<uint64_t>((count + kThreads * 8 - 1) / (kThreads * 8), 152ull * 8);
    k_ham_chunk<R><<<blocks, kThreads, 0, st>>>(static_cast<const T*>(psi_slots), static_cast<T*>(lam), c, terms,
                                               nterms, accumulate ? 1 : 0);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dot(const void* A, const void* B, uint64_t count, double* partials, int nblocks, cudaStream_t st)
{
    using T = typename V2<R>::T;
    k_dot<R><<<nblocks, kThreads, 0, st>>>(static_cast<const T*>(A), static_cast<const T*>(B), count, partials);
    return cudaGetLastError();
}

#define SV_INST(R)                                                                                              \
    template cudaError_t launch_pauli_partials<R>(const void*, const void*, int, uint64_t, const PauliDev*, int, \
                                                  double*, int, cudaStream_t);                                  \
    template cudaError_t launch_energy_partials<R>(const void*, int, uint64_t, const PauliDev*, int, double*, int, \
                                                   cudaStream_t);                                                \
    template cudaError_t launch_energy_tiles<R>(const void*, int, uint64_t, const EnergyTiles&, const PauliDev*, \
                                                int, double*, int, int*, cudaStream_t);                         \
    template cudaError_t launch_gather<R>(const void*, const uint64_t*, const uint64_t*, uint64_t, double*,     \
                                          cudaStream_t);                                                        \
    template cudaError_t launch_hamiltonian<R>(const void*, void*, int, const PauliDev*, int, cudaStream_t);    \
    template cudaError_t launch_dot<R>(const void*, const void*, uint64_t, double*, int, cudaStream_t);     \
    template cudaError_t launch_ham_chunk<R>(const void*, void*, int, const PauliDev*, int, bool, cudaStream_t);
SV_INST(float)
SV_INST(double)
#undef SV_INST

}  // namespace sv
