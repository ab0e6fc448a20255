// engine.cpp -- execution of planned passes (MEMQSim Sec. 2, "Online stage").
//
// Compressed mode: for each pass, chunk groups stream through a pipeline of
// pipeline_slots device buffers on three CUDA streams:
//   h2d  : compressed chunk streams, pinned host -> device (one bulk copy per
//          chunk, the paper's buffer strategy, Table 1)
//   comp : decode -> tile sub-passes -> encode, then the group's chunk sizes
//          device -> pinned host
//   d2h  : compressed chunk streams device -> pinned host, issued one group
//          later, once the sizes are on the host
// so that while group i is computed, group i+1 is copied in and group i-1
// copied out. Every chunk keeps one pinned slot: a pass writes the chunk's
// new stream over its old one (or into a larger slot when it grew), after
// the group's copy of the old stream to the device has completed.
// Uncompressed mode keeps the whole state in HBM and runs the sub-passes
// over it directly.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>

#include "engine.h"
#include "jit.h"

namespace sv {

// ------------------------------------------------------------------ errors
int fail(sv_state* s, int code, const std::string& msg)
{
    if (s) s->err = msg;
    return code;
}

int cuda_fail(sv_state* s, cudaError_t e, const char* where)
{
    return fail(s, SV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int wait_event(sv_state* s, cudaEvent_t ev)
{
    const auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) {
            s->st.t_host_wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            return SV_OK;
        }
        if (e != cudaErrorNotReady) return cuda_fail(s, e, "cudaEventQuery");
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > s->cfg.timeout_s) return fail(s, SV_ERR_TIMEOUT, "timed out waiting for GPU work");
    }
}

int wait_stream(sv_state* s, cudaStream_t st)
{
    const auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) {
            s->st.t_host_wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            return SV_OK;
        }
        if (e != cudaErrorNotReady) return cuda_fail(s, e, "cudaStreamQuery");
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > s->cfg.timeout_s) return fail(s, SV_ERR_TIMEOUT, "timed out waiting for GPU work");
    }
}

int sync_all(sv_state* s)
{
    int r;
    if ((r = wait_stream(s, s->s_h2d))) return r;
    if ((r = wait_stream(s, s->s_comp))) return r;
    if ((r = wait_stream(s, s->s_d2h))) return r;
    return SV_OK;
}

// read and clear the device error word
int check_device_error(sv_state* s)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->s_comp);
    if (e != cudaSuccess) return cuda_fail(s, e, "read error word");
    int r = wait_stream(s, s->s_comp);
    if (r) return r;
    if (h) {
        cudaMemsetAsync(s->d_err, 0, sizeof(int), s->s_comp);
        wait_stream(s, s->s_comp);
        if (h & kErrCorrupt) return fail(s, SV_ERR_CORRUPT, "compressed chunk stream failed validation");
        if (h & kErrRange) return fail(s, SV_ERR_RANGE, "amplitude outside the quantiser range or not finite");
        if (h & kErrWait) return fail(s, SV_ERR_TIMEOUT, "a kernel's wait for its copies exceeded its limit");
    }
    return SV_OK;
}

// ------------------------------------------------------------------ store
static void pool_remove(HostPool& pool, std::map<uint8_t*, std::pair<size_t, int>>::iterator it)
{
    auto range = pool.free_by_size.equal_range(it->second.first);
    for (auto jt = range.first; jt != range.second; ++jt)
        if (jt->second == it->first) {
            pool.free_by_size.erase(jt);
            break;
        }
    pool.free_at.erase(it);
}

static void pool_insert(HostPool& pool, uint8_t* p, size_t bytes, int seg)
{
    pool.free_at[p] = {bytes, seg};
    pool.free_by_size.emplace(bytes, p);
}

// Return [p, p + bytes) of segment `seg` to the pool, merged with the free
// blocks that touch it in the same segment.
static void pool_release(HostPool& pool, uint8_t* p, size_t bytes, int seg)
{
    auto next = pool.free_at.lower_bound(p);
    if (next != pool.free_at.end() && next->first == p + bytes && next->second.second == seg) {
        bytes += next->second.first;
        pool_remove(pool, next);
    }
    auto it = pool.free_at.lower_bound(p);
    if (it != pool.free_at.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second.first == p && prev->second.second == seg) {
            p = prev->first;
            bytes += prev->second.first;
            pool_remove(pool, prev);
        }
    }
    pool_insert(pool, p, bytes, seg);
}

static int pool_segment_of(const HostPool& pool, const uint8_t* p)
{
    for (size_t i = 0; i < pool.segs.size(); i++)
        if (p >= pool.segs[i].ptr && p < pool.segs[i].ptr + pool.segs[i].cap) return (int)i;
    return -1;
}

// A slot of `want` bytes (or of at least `need` when only a smaller free
// block is left): best fit among the free blocks, split when the rest is
// worth keeping, else from a new segment of seg_bytes (only `want` when the
// host budget has no room for a whole one). nullptr when the budget or the
// host is exhausted.
static uint8_t* pool_alloc(sv_state* s, HostPool& pool, uint64_t need, uint64_t want, uint64_t& cap)
{
    auto it = pool.free_by_size.lower_bound(want);
    if (it == pool.free_by_size.end()) {
        it = pool.free_by_size.lower_bound(need);
        if (it != pool.free_by_size.end()) want = it->first;  // a block between need and want: all of it
    }
    if (it == pool.free_by_size.end()) {
        size_t segb = std::max<size_t>(pool.seg_bytes, want);
        const uint64_t budget = s->cfg.host_budget_bytes;
        if (budget && s->pinned_bytes + segb > budget) segb = want;
        if (budget && s->pinned_bytes + segb > budget) return nullptr;
        void* p = nullptr;
        if (cudaHostAlloc(&p, segb, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        s->pinned_bytes += segb;
        pool.segs.push_back({static_cast<uint8_t*>(p), segb});
        pool_insert(pool, static_cast<uint8_t*>(p), segb, (int)pool.segs.size() - 1);
        it = pool.free_by_size.lower_bound(want);
    }
    uint8_t* p = it->second;
    auto at = pool.free_at.find(p);
    const size_t have = at->second.first;
    const int seg = at->second.second;
    pool_remove(pool, at);
    if (have - want >= 4096) {
        pool_insert(pool, p + want, have - want, seg);
        cap = want;
    } else {
        cap = have;
    }
    return p;
}

uint8_t* store_slot(sv_state* s, HostPool& pool, ChunkRef& ref, uint64_t bytes)
{
    if (ref.ptr && bytes <= ref.cap) {
        ref.bytes = bytes;
        return ref.ptr;
    }
    const uint64_t need = (bytes + 255) & ~uint64_t(255);
    const uint64_t want = (bytes + bytes / 32 + 255) & ~uint64_t(255);
    // Release the old slot first, so that it can merge into the block the new
    // one comes from: its stream has reached the device already, and a copy
    // still writing it (an earlier pass's, on the device-to-host stream)
    // precedes every later write into the region on that stream. A slot of
    // capacity 0 is the shared one and stays.
    if (ref.ptr && ref.cap) pool_release(pool, ref.ptr, ref.cap, pool_segment_of(pool, ref.ptr));
    uint64_t cap = 0;
    uint8_t* p = pool_alloc(s, pool, need, want, cap);
    ref = p ? ChunkRef{p, bytes, cap} : ChunkRef{};
    return p;
}

void store_release_all(HostPool& pool, std::vector<ChunkRef>& refs)
{
    for (ChunkRef& r : refs) {
        if (r.ptr && r.cap) pool_release(pool, r.ptr, r.cap, pool_segment_of(pool, r.ptr));
        r = ChunkRef{};
    }
    if (pool.shared) pool_release(pool, pool.shared, pool.shared_cap, pool_segment_of(pool, pool.shared));
    pool.shared = nullptr;
    pool.shared_cap = 0;
}

void pool_free(HostPool& pool)
{
    for (auto& g : pool.segs) cudaFreeHost(g.ptr);
    pool.segs.clear();
    pool.free_at.clear();
    pool.free_by_size.clear();
    pool.shared = nullptr;
    pool.shared_cap = 0;
}

// ------------------------------------------------------------- profiling
// With sv_config.profile, kernel launches on the compute stream are bracketed
// by CUDA events; durations are read once the pass has synchronised.
enum { PROF_DECODE = 0, PROF_APPLY = 1, PROF_ENCODE = 2, PROF_FINISH = 3, PROF_H2D = 4, PROF_D2H = 5 };

static int prof_begin(sv_state* s, cudaStream_t st = nullptr)
{
    if (!s->cfg.profile) return -1;
    if (!st) st = s->s_comp;
    const size_t i = s->prof_used;
    while (s->prof_ev.size() < 2 * (i + 1)) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return -1;
        s->prof_ev.push_back(ev);
    }
    if (s->prof_rec.size() < i + 1) s->prof_rec.resize(i + 1);
    cudaEventRecord(s->prof_ev[2 * i], st);
    s->prof_used++;
    return (int)i;
}

static void prof_end(sv_state* s, int i, int kind, uint64_t bytes, cudaStream_t st = nullptr)
{
    if (i < 0) return;
    cudaEventRecord(s->prof_ev[2 * i + 1], st ? st : s->s_comp);
    s->prof_rec[i] = {kind, bytes};
}

static void prof_collect(sv_state* s)
{
    for (size_t i = 0; i < s->prof_used; i++) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, s->prof_ev[2 * i], s->prof_ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const auto& r = s->prof_rec[i];
        if (r.kind == PROF_DECODE) { s->st.t_decode_s += ms * 1e-3; s->st.n_decode++; s->st.alg_bytes_decode += r.bytes; }
        if (r.kind == PROF_APPLY) { s->st.t_apply_s += ms * 1e-3; s->st.n_apply++; s->st.alg_bytes_apply += r.bytes; }
        if (r.kind == PROF_ENCODE) { s->st.t_encode_s += ms * 1e-3; s->st.n_encode++; s->st.alg_bytes_encode += r.bytes; }
        if (r.kind == PROF_FINISH) s->st.t_encode_finish_s += ms * 1e-3;
        if (r.kind == PROF_H2D) s->st.t_h2d_s += ms * 1e-3;
        if (r.kind == PROF_D2H) s->st.t_d2h_s += ms * 1e-3;
    }
    s->prof_used = 0;
}

// ----------------------------------------------------------- op upload
// Copy a pass's op tables (concatenated, 256-byte aligned sections) to the
// device buffer d_ops on the compute stream, growing the buffer if needed.
static int upload_blob(sv_state* s, const std::vector<uint8_t>& blob)
{
    const size_t bytes = std::max<size_t>(1, blob.size());
    if (bytes > s->ops_cap) {
        if (s->d_ops) {
            wait_stream(s, s->s_comp);
            dev_free(s, s->d_ops);
            s->d_ops = nullptr;
        }
        size_t cap = std::max<size_t>(bytes * 2, 1 << 16);
        cudaError_t e = dev_alloc(s, &s->d_ops, cap);
        if (e != cudaSuccess) return cuda_fail(s, e, "cudaMalloc(ops)");
        s->ops_cap = cap;
    }
    if (!blob.empty()) {
        cudaError_t e = cudaMemcpyAsync(s->d_ops, blob.data(), blob.size(), cudaMemcpyHostToDevice, s->s_comp);
        if (e != cudaSuccess) return cuda_fail(s, e, "upload ops");
    }
    return SV_OK;
}

template <typename V>
static size_t append_section(std::vector<uint8_t>& blob, const std::vector<V>& v)
{
    const size_t off = (blob.size() + 255) & ~size_t(255);
    blob.resize(off + v.size() * sizeof(V));
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(V));
    return off;
}

template <typename R>
int upload_ops(sv_state* s, const std::vector<DevOp<R>>& ops)
{
    std::vector<uint8_t> blob;
    append_section(blob, ops);
    return upload_blob(s, blob);
}

// Device form of a pass: every sub-pass's tile descriptor and its op range,
// as generic shared-memory ops or, on 2^12 tiles, as register phases.
template <typename R>
struct DevPass {
    std::vector<TileDesc> td;
    std::vector<int> off, cnt;
    std::vector<DevOp<R>> ops;
    bool use_phases = false;
    bool const_tables = false; // phase / op tables uploaded to constant memory
    bool fuse_decode = false;  // first sub-pass decodes the chunk streams
    bool fuse_encode = false;  // last sub-pass encodes the block pairs
    std::vector<int> ph_off, ph_cnt;
    std::vector<Phase> phases;
    std::vector<PhaseOp<R>> pops;
    std::vector<CtaCtrl> ctl;
    std::vector<R> d2m;
    size_t ops_at = 0, phases_at = 0, pops_at = 0, ctl_at = 0, d2m_at = 0;  // byte offsets in the uploaded blob
    // sub-pass kernels generated for this pass's gate sequences (jit.cpp), with
    // the matrix values each reads; a null kernel runs the table-driven one
    std::vector<const JitFn*> jfn;
    std::vector<std::vector<R>> jpar;
};

// Generate and compile (one parallel batch, cached per process) the
// specialised kernels of every register-phase sub-pass of `dps`.
template <typename R>
static int jit_prepare(sv_state* s, const std::vector<DevPass<R>*>& dps)
{
    if (!s->cfg.jit) return SV_OK;
    std::vector<std::string> keys;
    std::vector<std::pair<DevPass<R>*, size_t>> where;
    for (DevPass<R>* dp : dps) {
        if (!dp->use_phases) continue;
        const size_t ns = dp->td.size();
        dp->jfn.assign(ns, nullptr);
        dp->jpar.assign(ns, std::vector<R>());
        for (size_t i = 0; i < ns; i++) {
            const bool dec = i == 0 && dp->fuse_decode, enc = i + 1 == ns && dp->fuse_encode;
            const Phase* ph = dp->phases.data() + dp->ph_off[i];
            jit_params<R>(ph, dp->ph_cnt[i], dp->pops.data(), dp->d2m.data(), dp->jpar[i]);
            std::string key;
            jit_key<R>(ph, dp->ph_cnt[i], dp->pops.data(), dp->ctl.data(), dp->jpar[i], dec, enc, dp->td[i], key);
            keys.push_back(std::move(key));
            where.push_back({dp, i});
        }
    }
    if (keys.empty()) return SV_OK;
    auto source_of = [&](size_t k) {
        DevPass<R>* dp = where[k].first;
        const size_t i = where[k].second;
        return jit_source<R>(dp->phases.data() + dp->ph_off[i], dp->ph_cnt[i], dp->pops.data(), dp->ctl.data(),
                             dp->d2m.data(), i == 0 && dp->fuse_decode, i + 1 == dp->td.size() && dp->fuse_encode,
                             dp->td[i], dp->jpar[i]);
    };
    std::vector<const JitFn*> fns;
    std::string err;
    JitReport rep;
    if (!jit_compile(keys, source_of, s->cfg.device, fns, err, &rep))
        return fail(s, SV_ERR_CUDA, "run-time kernel compilation failed: " + err);
    for (size_t k = 0; k < keys.size(); k++) where[k].first->jfn[where[k].second] = fns[k];
    s->st.jit_kernels_compiled += rep.compiled;
    s->st.t_jit_compile_s += rep.seconds;
    return SV_OK;
}

template <typename R>
static DevPass<R> build_dev_pass(const std::vector<SubPlan>& subs, int L, int t, int l, bool fuse_decode = false,
                                 bool fuse_encode = false)
{
    DevPass<R> dp;
    dp.use_phases = (t == kPhaseTileQubits && l >= 4 && l <= 5);
    dp.fuse_decode = dp.use_phases && fuse_decode;
    dp.fuse_encode = dp.use_phases && fuse_encode;
    for (size_t si = 0; si < subs.size(); si++) {
        const SubPlan& sp = subs[si];
        // sub-passes that fuse the codec use rows of whole block pairs (l = 8)
        const bool codec_rows = dp.use_phases && ((si == 0 && dp.fuse_decode) || (si + 1 == subs.size() && dp.fuse_encode));
        TileDesc td = tile_desc(sp.T, L, t, codec_rows ? 8 : l);
        if (dp.use_phases) order_tile_bits<R>(sp, td, false);
        dp.td.push_back(td);
        dp.off.push_back((int)dp.ops.size());
        dp.ph_off.push_back((int)dp.phases.size());
        if (dp.use_phases) dev_phases<R>(sp, td, dp.phases, dp.pops, dp.ctl, dp.d2m);
        else dev_ops<R>(sp, td, dp.ops, nullptr, nullptr);
        dp.cnt.push_back((int)dp.ops.size() - dp.off.back());
        dp.ph_cnt.push_back((int)dp.phases.size() - dp.ph_off.back());
    }
    return dp;
}

template <typename R>
static int upload_pass(sv_state* s, DevPass<R>& dp)
{
    // generated kernels take their matrices by value: nothing to upload (the
    // copy from pageable host memory would wait for the compute stream)
    bool all_generated = dp.use_phases && !dp.jfn.empty();
    for (const JitFn* f : dp.jfn)
        if (!f) all_generated = false;
    if (all_generated) return SV_OK;
    std::vector<uint8_t> blob;
    dp.ops_at = append_section(blob, dp.ops);
    dp.phases_at = append_section(blob, dp.phases);
    dp.pops_at = append_section(blob, dp.pops);
    dp.ctl_at = append_section(blob, dp.ctl);
    dp.d2m_at = append_section(blob, dp.d2m);
    int r = upload_blob(s, blob);
    if (r) return r;
    // phase / op tables also go to constant memory when they fit (uniform dispatch)
    dp.const_tables = dp.use_phases && upload_const_tables<R>(dp.phases.data(), (int)dp.phases.size(),
                                                              dp.pops.data(), (int)dp.pops.size(), s->s_comp);
    return SV_OK;
}

// Adjoint sub-passes as generated two-vector kernels (jit.cpp): psi and
// lambda in registers, the gradient partials inline. `ok` stays false (the
// k_adjoint path runs) when generation is off or a sub-pass cannot be
// specialised; the sub-passes' gradient slots are then left to that path.
template <typename R>
struct AdjPlan {
    bool ok = false;
    std::vector<TileDesc> td;
    std::vector<std::vector<R>> par;
    std::vector<const JitFn*> fn;
    std::vector<int> nsl, gslot;  // gradient slots of each sub-pass, index of its first one in slot_params
};

template <typename R>
static int jit_adjoint_plan(sv_state* s, const std::vector<SubPlan>& subs, int L, int t, int l,
                            std::vector<int>& slot_params, AdjPlan<R>& ap)
{
    ap = AdjPlan<R>();
    if (!s->cfg.jit || t != kPhaseTileQubits || l < 4 || l > 5 || subs.empty()) return SV_OK;
    struct Sub {
        std::vector<Phase> ph;
        std::vector<PhaseOp<R>> ops;
        std::vector<CtaCtrl> ctl;
        std::vector<R> d2m;
        std::vector<int32_t> grad;
    };
    std::vector<Sub> sv(subs.size());
    std::vector<int> sp_local;
    std::vector<std::string> keys(subs.size());
    for (size_t i = 0; i < subs.size(); i++) {
        TileDesc td = tile_desc(subs[i].T, L, t, l);
        order_tile_bits<R>(subs[i], td, true);
        ap.td.push_back(td);
        ap.gslot.push_back((int)(slot_params.size() + sp_local.size()));
        const size_t before = sp_local.size();
        dev_phases<R>(subs[i], td, sv[i].ph, sv[i].ops, sv[i].ctl, sv[i].d2m, &sv[i].grad, &sp_local);
        ap.nsl.push_back((int)(sp_local.size() - before));
        ap.par.emplace_back();
        jit_params<R>(sv[i].ph.data(), (int)sv[i].ph.size(), sv[i].ops.data(), sv[i].d2m.data(), ap.par.back(), false);
        jit_key<R>(sv[i].ph.data(), (int)sv[i].ph.size(), sv[i].ops.data(), sv[i].ctl.data(), ap.par.back(), false,
                   false, td, keys[i], sv[i].grad.data());
    }
    auto source_of = [&](size_t k) {
        return jit_source<R>(sv[k].ph.data(), (int)sv[k].ph.size(), sv[k].ops.data(), sv[k].ctl.data(),
                             sv[k].d2m.data(), false, false, ap.td[k], ap.par[k], sv[k].grad.data());
    };
    std::string err;
    JitReport rep;
    if (!jit_compile(keys, source_of, s->cfg.device, ap.fn, err, &rep))
        return fail(s, SV_ERR_CUDA, "run-time kernel compilation failed: " + err);
    s->st.jit_kernels_compiled += rep.compiled;
    s->st.t_jit_compile_s += rep.seconds;
    for (const JitFn* f : ap.fn)
        if (!f) return SV_OK;
    slot_params.insert(slot_params.end(), sp_local.begin(), sp_local.end());
    ap.ok = true;
    return SV_OK;
}

// launch sub-pass i of an uploaded pass on a buffer of 2^L local amplitudes
template <typename R>
static cudaError_t launch_subpass(sv_state* s, const DevPass<R>& dp, size_t i, void* amps, uint64_t gbase,
                                  const FuseArgs* fa = nullptr)
{
    const uint8_t* base = static_cast<const uint8_t*>(s->d_ops);
    static const FuseArgs none{};
    if (dp.use_phases && i < dp.jfn.size() && dp.jfn[i]) {
        s->st.jit_launches++;
        return jit_launch<R>(dp.jfn[i], amps, dp.td[i], gbase, fa ? *fa : none, dp.jpar[i], s->s_comp);
    }
    if (dp.use_phases) {
        const int p0 = dp.ph_off[i], pn = dp.ph_cnt[i];
        const int op0 = pn ? dp.phases[p0].op_begin : 0;
        const int nops = pn ? dp.phases[p0 + pn - 1].op_begin + dp.phases[p0 + pn - 1].op_count - op0 : 0;
        return launch_apply_phases<R>(amps, dp.td[i], reinterpret_cast<const Phase*>(base + dp.phases_at) + p0, pn,
                                      reinterpret_cast<const PhaseOp<R>*>(base + dp.pops_at), op0, nops,
                                      reinterpret_cast<const CtaCtrl*>(base + dp.ctl_at),
                                      reinterpret_cast<const R*>(base + dp.d2m_at), gbase, fa ? *fa : none, s->s_comp,
                                      dp.const_tables ? p0 : -1);
    }
    return launch_apply<R>(amps, dp.td[i], reinterpret_cast<const DevOp<R>*>(base + dp.ops_at) + dp.off[i], dp.cnt[i],
                           gbase, s->s_comp);
}

// Tile shape over L local positions: t tile qubits of which the low l are
// always included; at least two tile positions stay free for the mixing
// targets of a gate unless the tile covers every local position.
void tile_shape(int L, int tq, int lq, int& t, int& l)
{
    t = std::min(tq, L);
    if (t < L) {
        t = std::min(L, std::max(t, 3));
        l = std::max(1, std::min(lq, t - 2));
    } else {
        l = std::max(1, std::min(lq, t));
    }
}

static inline uint64_t deposit(uint64_t v, const std::vector<int>& pos)
{
    uint64_t r = 0;
    for (size_t i = 0; i < pos.size(); i++)
        if ((v >> i) & 1) r |= 1ull << pos[i];
    return r;
}

// --------------------------------------------------- compressed streaming
// Plan one pass for the device: its tile sub-passes, whether the codec
// fuses into the first / last of them, and their device form.
template <typename R>
static int prepare_pass_compressed(const sv_state* s, const std::vector<PGate>& gates, const PassPlan& pp,
                                   DevPass<R>& dp, std::string& err)
{
    const int c = s->c, g = (int)pp.S.size();
    const int L = c + g;
    int t, l;
    tile_shape(L, s->tq, s->lq, t, l);
    const std::vector<HOp> hops = local_ops(gates, pp.gates, c, pp.S, false);
    std::vector<SubPlan> subs = plan_subpasses(hops, L, t, l, true);
    if (subs.empty() && !hops.empty()) {
        err = "no tile plan for the pass";
        return SV_ERR_ARG;
    }
    // Fuse the decode into the first sub-pass when a plan whose first tile
    // holds whole block pairs (local bits 0..7) needs no extra sub-pass, and
    // the encode into the last sub-pass when its tile holds them.
    bool fdec = false, fenc = false;
    // (the relative bound's step needs the chunk maximum before any block is encoded)
    if (t == kPhaseTileQubits && l >= 4 && l <= 5 && c >= 8 && !subs.empty() && s->cfg.fuse_codec && !s->rel) {
        std::vector<SubPlan> alt = plan_subpasses(hops, L, t, l, true, 8);
        if (!alt.empty() && alt.size() <= subs.size()) {
            subs.swap(alt);
            fdec = true;
        }
        fenc = replan_tail(subs, L, t, l, 8, fdec);
    }
    dp = build_dev_pass<R>(subs, L, t, l, fdec, fenc);
    return SV_OK;
}

// Stream every chunk group of the passes through the GPU (Sec. 2, "Online
// stage" steps (1)-(6)): per group, host -> device copies of its chunk
// streams, decode, the pass's tile sub-passes, encode, device -> host copies.
// Group issues run one ahead of their completions, across pass boundaries
// too: the next pass's first copies overlap the previous pass's last group,
// whose streams the next pass takes from the device (copied into d_carry by a
// kernel right after their encode) instead of through the host.
template <typename R>
static int stream_passes(sv_state* s, const std::vector<PassPlan>& passes, std::vector<DevPass<R>>& dps)
{
    const int c = s->c, NS = s->nslots;
    struct PassInfo {
        std::vector<int> spos, fpos;  // chunk-index bit positions of staged and fixed high qubits
        uint64_t ngroups = 0, done = 0;
        int g = 0, gch = 0, L = 0;
        double norm2 = 0;
    };
    std::vector<PassInfo> pinfo(passes.size());
    std::vector<std::pair<int, uint64_t>> items;  // (pass, group) in issue order
    for (size_t p = 0; p < passes.size(); p++) {
        PassInfo& P = pinfo[p];
        for (int q = c; q < s->n; q++) {
            if (std::find(passes[p].S.begin(), passes[p].S.end(), q) != passes[p].S.end()) P.spos.push_back(q - c);
            else P.fpos.push_back(q - c);
        }
        P.g = (int)passes[p].S.size();
        P.gch = 1 << P.g;
        P.L = c + P.g;
        P.ngroups = 1ull << P.fpos.size();
        for (uint64_t gi = 0; gi < P.ngroups; gi++) items.push_back({(int)p, gi});
    }
    // renormalisation feeds a pass's norm into the next pass's decode: no
    // lookahead across passes then
    const bool cross = !s->cfg.renormalize;
    std::vector<std::vector<uint64_t>> slot_chunks(NS);
    std::vector<int> slot_prof(NS, -1);
    std::vector<std::pair<uint64_t, int>> carry_next;  // chunks the current pass leaves in d_carry
    std::vector<uint64_t> unsized;                      // carried chunks of the group being issued, length unknown
    std::vector<std::pair<int, std::vector<uint64_t>>> unsized_prof;  // profiled launches reading them
    for (int32_t& v : s->carry_at) v = -1;

    auto issue = [&](size_t idx) -> int {
        const int p = items[idx].first;
        const uint64_t gi = items[idx].second;
        PassInfo& P = pinfo[p];
        DevPass<R>& dp = dps[p];
        const int slot = (int)(idx % NS), gch = P.gch, L = P.L;
        cudaError_t e;
        int r;
        if (gi == 0) {
            // this pass reads the previous pass's last group from d_carry and
            // its other groups from the host once their copies are complete
            for (int32_t& v : s->carry_at) v = -1;
            for (const auto& kj : carry_next) s->carry_at[kj.first] = kj.second;
            carry_next.clear();
            if (p > 0 && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_prev_d2h, 0))) return cuda_fail(s, e, "wait d2h");
            if ((r = upload_pass<R>(s, dp))) return r;
        }
        const uint64_t base = deposit(gi, P.fpos);
        auto& ch = slot_chunks[slot];
        ch.resize(gch);
        GroupIn gin{};
        StreamMoves mv;
        if (s->slot_used[slot] && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_comp[slot], 0)))
            return cuda_fail(s, e, "wait comp");
        const int ph2d = prof_begin(s, s->s_h2d);
        for (int j = 0; j < gch; j++) {
            const uint64_t k = base | deposit((uint64_t)j, P.spos);
            ch[j] = k;
            if (s->carry_at[k] >= 0) {
                // on the device: gathered into the slot by a kernel below. Before
                // the previous pass's last group completes on the host its length
                // is known on the device only: decode then bounds it by the slot
                mv.src[mv.n] = (uint16_t)s->carry_at[k];
                mv.dst[mv.n] = (uint16_t)j;
                mv.n++;
                if (p > 0 && pinfo[p - 1].done == pinfo[p - 1].ngroups) {
                    gin.bytes[j] = (uint32_t)s->cur[k].bytes;
                } else {
                    gin.bytes[j] = (uint32_t)s->stride;
                    unsized.push_back(k);
                }
                continue;
            }
            const ChunkRef& cr = s->cur[k];
            gin.bytes[j] = (uint32_t)cr.bytes;
            if ((e = cudaMemcpyAsync(s->d_in[slot] + (size_t)j * s->stride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice,
                                     s->s_h2d)))
                return cuda_fail(s, e, "H2D chunk");
            s->st.bytes_h2d += cr.bytes;
        }
        prof_end(s, ph2d, PROF_H2D, 0, s->s_h2d);
        if ((e = cudaEventRecord(s->ev_h2d[slot], s->s_h2d))) return cuda_fail(s, e, "record h2d");
        if ((e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[slot], 0))) return cuda_fail(s, e, "wait h2d");
        if (s->slot_used[slot] && (e = cudaStreamWaitEvent(s->s_comp, s->ev_d2h[slot], 0)))
            return cuda_fail(s, e, "wait d2h");
        if (mv.n && (e = launch_gather_streams(s->d_carry, s->d_carry_bytes, s->stride, s->d_in[slot], s->stride, mv, s->s_comp)))
            return cuda_fail(s, e, "gather streams");
        if (mv.n) s->st.kernel_launches++;
        const uint64_t amp_bytes = (sizeof(R) * 2ull) << L;
        uint64_t in_bytes = 0;
        for (int j = 0; j < gch; j++) in_bytes += gin.bytes[j];
        in_bytes -= (uint64_t)unsized.size() * s->stride;  // their lengths are added once known
        int pi = -1;
        if (!dp.fuse_decode) {
            pi = prof_begin(s);
            if ((e = launch_decode<R>(s->d_in[slot], s->stride, c, s->dtype, gch, gin, s->d_amps, s->scale, s->d_err,
                                      s->s_comp)))
                return cuda_fail(s, e, "decode");
            prof_end(s, pi, PROF_DECODE, in_bytes + amp_bytes);
            if (!unsized.empty()) unsized_prof.push_back({pi, unsized});
            s->st.kernel_launches++;
        }
        const uint64_t gbase = base << c;
        FuseArgs fa;
        fa.c = c;
        fa.dtype = s->dtype;
        fa.k = s->k;
        fa.scale = s->scale;
        fa.in = s->d_in[slot];
        fa.in_stride = s->stride;
        fa.gin = gin;
        fa.out = s->d_out[slot];
        fa.out_stride = s->stride;
        fa.sparse = s->d_sparse;
        fa.blocksq = s->d_blocksq;
        fa.err = s->d_err;
        slot_prof[slot] = -1;
        for (size_t i = 0; i < dp.td.size(); i++) {
            fa.decode = (i == 0 && dp.fuse_decode) ? 1 : 0;
            fa.encode = (i + 1 == dp.td.size() && dp.fuse_encode) ? 1 : 0;
            pi = prof_begin(s);
            if ((e = launch_subpass<R>(s, dp, i, s->d_amps, gbase, &fa))) return cuda_fail(s, e, "apply");
            // algorithmic bytes: what the launch reads (stream or amplitudes) and writes
            // (amplitudes; a fused encode's stream bytes are added once known)
            prof_end(s, pi, PROF_APPLY, (fa.decode ? in_bytes : amp_bytes) + (fa.encode ? 0 : amp_bytes));
            if (fa.decode && !unsized.empty()) unsized_prof.push_back({pi, unsized});
            if (fa.encode) slot_prof[slot] = pi;
            s->st.kernel_launches++;
        }
        unsized.clear();
        int launches = 0;
        if (dp.fuse_encode) {
            const int pf = prof_begin(s);
            if ((e = launch_encode_finish(c, s->dtype, s->k, gch, s->d_out[slot], s->stride, s->d_sparse, s->d_blocksq,
                                          s->d_co[slot], s->s_comp, &launches)))
                return cuda_fail(s, e, "encode");
            prof_end(s, pf, PROF_FINISH, 0);
        } else {
            pi = prof_begin(s);
            slot_prof[slot] = pi;
            if (s->rel && (e = launch_chunk_steps<R>(s->d_amps, c, gch, s->eb, s->d_mbits, s->d_kc, s->s_comp,
                                                     &launches)))
                return cuda_fail(s, e, "chunk steps");
            if ((e = launch_encode<R>(s->d_amps, c, s->dtype, s->k, gch, s->d_out[slot], s->stride, s->d_sparse,
                                      s->d_blocksq, s->d_co[slot], s->d_err, s->s_comp, &launches,
                                      s->rel ? s->d_kc : nullptr)))
                return cuda_fail(s, e, "encode");
            prof_end(s, pi, PROF_ENCODE, amp_bytes);
        }
        s->st.kernel_launches += launches;
        if (cross && gi + 1 == P.ngroups && (size_t)p + 1 < passes.size()) {
            // the last group of a pass: its streams stay on the device for the next pass
            if ((e = launch_copy_streams(s->d_out[slot], s->d_co[slot], s->d_carry, s->d_carry_bytes, s->stride, gch,
                                         s->s_comp)))
                return cuda_fail(s, e, "carry streams");
            s->st.kernel_launches++;
            for (int j = 0; j < gch; j++) carry_next.push_back({ch[j], j});
        }
        if ((e = cudaMemcpyAsync(s->h_co[slot], s->d_co[slot], sizeof(ChunkOut) * gch, cudaMemcpyDeviceToHost,
                                 s->s_comp)))
            return cuda_fail(s, e, "D2H sizes");
        if ((e = cudaEventRecord(s->ev_comp[slot], s->s_comp))) return cuda_fail(s, e, "record comp");
        s->slot_used[slot] = true;
        s->st.groups++;
        s->st.subpasses += dp.td.size();
        return SV_OK;
    };

    auto finish = [&](size_t idx) -> int {
        const int p = items[idx].first;
        PassInfo& P = pinfo[p];
        const int slot = (int)(idx % NS), gch = P.gch;
        int rr = wait_event(s, s->ev_comp[slot]);
        if (rr) return rr;
        cudaError_t e;
        // the group's copies of its chunks' previous streams to the device are
        // complete (the compute event waited on them): their slots can be rewritten
        const int pd2h = prof_begin(s, s->s_d2h);
        for (int j = 0; j < gch; j++) {
            const uint64_t k = slot_chunks[slot][j];
            const ChunkOut co = s->h_co[slot][j];
            if (co.bytes > s->stride) return fail(s, SV_ERR_CORRUPT, "encoded chunk larger than its slot");
            uint8_t* dst = store_slot(s, s->pool, s->cur[k], co.bytes);
            if (!dst) return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the compressed store failed");
            if ((e = cudaMemcpyAsync(dst, s->d_out[slot] + (size_t)j * s->stride, co.bytes, cudaMemcpyDeviceToHost,
                                     s->s_d2h)))
                return cuda_fail(s, e, "D2H chunk");
            s->st.bytes_d2h += co.bytes;
            if (slot_prof[slot] >= 0) s->prof_rec[slot_prof[slot]].bytes += co.bytes;
            P.norm2 += (double)co.sumsq * std::ldexp(1.0, 2 * co.k);
        }
        prof_end(s, pd2h, PROF_D2H, 0, s->s_d2h);
        if ((e = cudaEventRecord(s->ev_d2h[slot], s->s_d2h)) || (e = cudaEventRecord(s->ev_prev_d2h, s->s_d2h)))
            return cuda_fail(s, e, "record d2h");
        if (++P.done == P.ngroups) {
            // the streams this pass left on the device now have their lengths
            for (const auto& u : unsized_prof)
                if (u.first >= 0)
                    for (uint64_t k : u.second) s->prof_rec[u.first].bytes += s->cur[k].bytes;
            unsized_prof.clear();
            s->st.passes++;
            s->st.norm2 = P.norm2;
            if (P.norm2 < 1e-300) return fail(s, SV_ERR_NORM_COLLAPSE, "norm of the stored state collapsed to zero");
            s->scale = s->cfg.renormalize ? 1.0 / std::sqrt(P.norm2) : 1.0;
        }
        return SV_OK;
    };

    int r = SV_OK;
    for (size_t idx = 0; idx <= items.size() && !r; idx++) {
        // without lookahead across passes, a pass's last group completes before the next pass starts
        const bool boundary = idx < items.size() && idx >= 1 && items[idx].first != items[idx - 1].first;
        if (!cross && boundary && (r = finish(idx - 1))) break;
        if (idx < items.size() && (r = issue(idx))) break;
        if (idx >= 1 && !(!cross && boundary) && (r = finish(idx - 1))) break;
    }
    const int rs = sync_all(s);
    for (int32_t& v : s->carry_at) v = -1;
    if (r) return r;
    if (rs) return rs;
    prof_collect(s);
    if ((r = check_device_error(s))) return r;
    uint64_t total = 0;
    for (const ChunkRef& cr : s->cur) total += cr.bytes;
    s->st.compressed_bytes = total;
    return SV_OK;
}

template <typename R>
int run_pass_compressed(sv_state* s, const std::vector<PGate>& gates, const PassPlan& pp)
{
    std::vector<DevPass<R>> dps(1);
    std::string err;
    int r = prepare_pass_compressed<R>(s, gates, pp, dps[0], err);
    if (r) return fail(s, r, err);
    r = jit_prepare<R>(s, {&dps[0]});
    if (!r) r = stream_passes<R>(s, {pp}, dps);
    return r;
}

// ------------------------------------------------------------ uncompressed
template <typename R>
int run_pass_uncompressed(sv_state* s, void* state, const std::vector<PGate>& gates, const std::vector<int>& ids)
{
    const int L = s->n;
    int t, l;
    tile_shape(L, s->tq, s->lq, t, l);
    const std::vector<int> noS;
    const std::vector<HOp> hops = local_ops(gates, ids, L, noS, false);
    const std::vector<SubPlan> subs = plan_subpasses(hops, L, t, l, true);
    if (subs.empty() && !hops.empty()) return fail(s, SV_ERR_ARG, "no tile plan for the pass");
    DevPass<R> dp = build_dev_pass<R>(subs, L, t, l);
    int r = jit_prepare<R>(s, {&dp});
    if (r) return r;
    if ((r = upload_pass<R>(s, dp))) return r;
    const uint64_t amp_bytes = (sizeof(R) * 2ull) << L;
    for (size_t i = 0; i < dp.td.size(); i++) {
        const int pi = prof_begin(s);
        cudaError_t e = launch_subpass<R>(s, dp, i, state, 0);
        if (e) return cuda_fail(s, e, "apply");
        prof_end(s, pi, PROF_APPLY, 2 * amp_bytes);
        s->st.kernel_launches++;
    }
    s->st.subpasses += dp.td.size();
    s->st.passes++;
    r = wait_stream(s, s->s_comp);
    prof_collect(s);
    return r;
}

template <typename R>
int apply_circuit(sv_state* s, const std::vector<PGate>& input, bool remap)
{
    if (input.empty()) return SV_OK;
    if (s->mode == SV_UNCOMPRESSED) {
        std::vector<int> ids(input.size());
        for (size_t i = 0; i < input.size(); i++) ids[i] = (int)i;
        return run_pass_uncompressed<R>(s, s->d_state, input, ids);
    }
    const auto t0 = std::chrono::steady_clock::now();
    // with remapping the passes run a gate list of their own (the input's
    // gates on moved positions plus physical SWAPs)
    std::vector<PGate> gates;
    std::vector<int> where;
    const std::vector<PassPlan> passes = plan_circuit(input, s->n, s->c, s->gmax, remap, gates, where);
    // plan every pass first, so that their kernels compile in one parallel batch
    std::vector<DevPass<R>> dps(passes.size());
    std::vector<DevPass<R>*> ptrs;
    {
        // passes are planned independently: one host thread each (bounded)
        std::vector<int> codes(passes.size(), SV_OK);
        std::vector<std::string> errs(passes.size());
        std::atomic<size_t> next{0};
        auto worker = [&]() {
            for (size_t i; (i = next.fetch_add(1)) < passes.size();)
                codes[i] = prepare_pass_compressed<R>(s, gates, passes[i], dps[i], errs[i]);
        };
        const size_t nth = std::min<size_t>(passes.size(), std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (size_t k = 1; k < nth; k++) pool.emplace_back(worker);
        worker();
        for (std::thread& th : pool) th.join();
        for (size_t i = 0; i < passes.size(); i++)
            if (codes[i]) return fail(s, codes[i], errs[i]);
        for (size_t i = 0; i < passes.size(); i++) ptrs.push_back(&dps[i]);
    }
    int r = jit_prepare<R>(s, ptrs);
    if (r) return r;
    s->st.t_host_prepare_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if ((r = stream_passes<R>(s, passes, dps))) return r;
    for (int& p : s->perm) p = where[p];  // logical qubits follow their moves
    s->st.remap_swaps += gates.size() - input.size();
    return SV_OK;
}

template <typename R>
int jit_sources(sv_state* s, const std::vector<PGate>& gates, std::vector<std::string>& out, bool adjoint)
{
    if (adjoint) {
        // the reverse sweep of sv_grad: every pass in reverse order, daggered gates
        std::vector<PGate> inv(gates.size());
        for (size_t i = 0; i < gates.size(); i++) {
            inv[i] = gates[i];
            const int K = 1 << gates[i].nt;
            for (int a = 0; a < K; a++)
                for (int b = 0; b < K; b++) inv[i].m[a * K + b] = std::conj(gates[i].m[b * K + a]);
        }
        std::vector<PassPlan> passes;
        if (s->mode == SV_UNCOMPRESSED) {
            PassPlan pp;
            for (size_t i = 0; i < gates.size(); i++) pp.gates.push_back((int)i);
            passes.push_back(pp);
        } else {
            passes = plan_passes(gates, s->n, s->c, s->gmax);
        }
        for (size_t p = passes.size(); p-- > 0;) {
            const PassPlan& pp = passes[p];
            const int c = s->mode == SV_UNCOMPRESSED ? s->n : s->c;
            const int L = c + (int)pp.S.size();
            int t, l;
            tile_shape(L, std::min(s->tq, 12), s->lq, t, l);
            if (t != kPhaseTileQubits || l < 4 || l > 5) continue;
            std::vector<int> rids(pp.gates.rbegin(), pp.gates.rend());
            const std::vector<SubPlan> subs = plan_subpasses(local_ops(inv, rids, c, pp.S, true), L, t, l, true);
            for (const SubPlan& sp : subs) {
                TileDesc td = tile_desc(sp.T, L, t, l);
                order_tile_bits<R>(sp, td, true);
                std::vector<Phase> ph;
                std::vector<PhaseOp<R>> ops;
                std::vector<CtaCtrl> ctl;
                std::vector<R> d2m, par;
                std::vector<int32_t> grad;
                std::vector<int> slots;
                dev_phases<R>(sp, td, ph, ops, ctl, d2m, &grad, &slots);
                jit_params<R>(ph.data(), (int)ph.size(), ops.data(), d2m.data(), par, false);
                out.push_back(jit_source<R>(ph.data(), (int)ph.size(), ops.data(), ctl.data(), d2m.data(), false,
                                            false, td, par, grad.data()));
            }
        }
        return SV_OK;
    }
    std::vector<DevPass<R>> dps;
    if (s->mode == SV_UNCOMPRESSED) {
        int t, l;
        tile_shape(s->n, s->tq, s->lq, t, l);
        std::vector<int> ids(gates.size());
        for (size_t i = 0; i < gates.size(); i++) ids[i] = (int)i;
        const std::vector<HOp> hops = local_ops(gates, ids, s->n, std::vector<int>(), false);
        const std::vector<SubPlan> subs = plan_subpasses(hops, s->n, t, l, true);
        if (subs.empty() && !hops.empty()) return fail(s, SV_ERR_ARG, "no tile plan for the pass");
        dps.push_back(build_dev_pass<R>(subs, s->n, t, l));
    } else {
        std::vector<PGate> rg;
        std::vector<int> where;
        const std::vector<PassPlan> passes =
            plan_circuit(gates, s->n, s->c, s->gmax, s->cfg.remap_qubits != 0, rg, where);
        dps.resize(passes.size());
        for (size_t i = 0; i < passes.size(); i++) {
            std::string err;
            int r = prepare_pass_compressed<R>(s, rg, passes[i], dps[i], err);
            if (r) return fail(s, r, err);
        }
    }
    for (DevPass<R>& dp : dps) {
        if (!dp.use_phases) continue;
        for (size_t i = 0; i < dp.td.size(); i++) {
            std::vector<R> par;
            const Phase* ph = dp.phases.data() + dp.ph_off[i];
            jit_params<R>(ph, dp.ph_cnt[i], dp.pops.data(), dp.d2m.data(), par);
            out.push_back(jit_source<R>(ph, dp.ph_cnt[i], dp.pops.data(), dp.ctl.data(), dp.d2m.data(),
                                        i == 0 && dp.fuse_decode, i + 1 == dp.td.size() && dp.fuse_encode,
                                        dp.td[i], par));
        }
    }
    return SV_OK;
}

// --------------------------------------------------------------- init
template <typename R>
int init_state(sv_state* s)
{
    cudaError_t e;
    const uint64_t init = s->cfg.init_index;
    if (s->mode == SV_UNCOMPRESSED) {
        if ((e = launch_fill_basis<R>(s->d_state, 1ull << s->n, (int64_t)init, s->s_comp)))
            return cuda_fail(s, e, "fill");
        s->st.kernel_launches++;
        s->st.norm2 = 1.0;
        return wait_stream(s, s->s_comp);
    }
    const int c = s->c;
    const uint64_t nchunks = 1ull << s->nh;
    const uint64_t cs = 1ull << c;
    // encode one all-zero chunk (slot 0) and the chunk holding the basis amplitude (slot 1)
    const int nenc = nchunks > 1 ? 2 : 1;
    if ((e = launch_fill_basis<R>(s->d_amps, cs * nenc, (int64_t)(nenc == 2 ? cs + (init & (cs - 1)) : init),
                                  s->s_comp)))
        return cuda_fail(s, e, "fill");
    int launches = 1;
    if (s->rel && (e = launch_chunk_steps<R>(s->d_amps, c, nenc, s->eb, s->d_mbits, s->d_kc, s->s_comp, &launches)))
        return cuda_fail(s, e, "chunk steps");
    if ((e = launch_encode<R>(s->d_amps, c, s->dtype, s->k, nenc, s->d_out[0], s->stride, s->d_sparse,
                              s->d_blocksq, s->d_co[0], s->d_err, s->s_comp, &launches, s->rel ? s->d_kc : nullptr)))
        return cuda_fail(s, e, "encode");
    s->st.kernel_launches += launches;
    if ((e = cudaMemcpyAsync(s->h_co[0], s->d_co[0], sizeof(ChunkOut) * nenc, cudaMemcpyDeviceToHost, s->s_comp)))
        return cuda_fail(s, e, "D2H sizes");
    int r = wait_stream(s, s->s_comp);
    if (r) return r;
    if ((r = check_device_error(s))) return r;
    std::vector<std::vector<uint8_t>> streams(nenc);
    for (int j = 0; j < nenc; j++) {
        streams[j].resize(s->h_co[0][j].bytes);
        if ((e = cudaMemcpy(streams[j].data(), s->d_out[0] + (size_t)j * s->stride, streams[j].size(),
                            cudaMemcpyDeviceToHost)))
            return cuda_fail(s, e, "D2H init stream");
        s->st.bytes_d2h += streams[j].size();
    }
    // every chunk but the basis amplitude's holds the same all-zero stream:
    // one shared slot (capacity 0, so the first pass that writes a chunk
    // gives it a slot of its own); earlier slots return to the pool
    const uint64_t init_chunk = init >> c;
    store_release_all(s->pool, s->cur);
    uint64_t total = 0;
    ChunkRef zero{};
    if (nenc == 2) {
        uint8_t* dst = store_slot(s, s->pool, zero, streams[0].size());
        if (!dst) return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the compressed store failed");
        std::memcpy(dst, streams[0].data(), streams[0].size());
        s->pool.shared = zero.ptr;
        s->pool.shared_cap = zero.cap;
        zero.cap = 0;
    }
    for (uint64_t k = 0; k < nchunks; k++) {
        if (nenc == 2 && k != init_chunk) {
            s->cur[k] = zero;
        } else {
            const std::vector<uint8_t>& src = streams[nenc - 1];
            uint8_t* dst = store_slot(s, s->pool, s->cur[k], src.size());
            if (!dst) return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the compressed store failed");
            std::memcpy(dst, src.data(), src.size());
        }
        total += s->cur[k].bytes;
    }
    s->st.compressed_bytes = total;
    s->st.norm2 = 1.0;
    s->scale = 1.0;
    return SV_OK;
}

// ----------------------------------------------------- read-only staging
// Stage chunks ks[0..m) (m <= 2^gmax) into d_amps slots 0..m-1 (decoded).
template <typename R>
int stage_chunks(sv_state* s, const std::vector<uint64_t>& ks)
{
    GroupIn gin{};
    cudaError_t e;
    const int m = (int)ks.size();
    for (int j = 0; j < m; j++) {
        const ChunkRef& cr = s->cur[ks[j]];
        gin.bytes[j] = (uint32_t)cr.bytes;
        if ((e = cudaMemcpyAsync(s->d_in[0] + (size_t)j * s->stride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice,
                                 s->s_comp)))
            return cuda_fail(s, e, "H2D chunk");
        s->st.bytes_h2d += cr.bytes;
    }
    if ((e = launch_decode<R>(s->d_in[0], s->stride, s->c, s->dtype, m, gin, s->d_amps, s->scale, s->d_err,
                              s->s_comp)))
        return cuda_fail(s, e, "decode");
    s->st.kernel_launches++;
    return SV_OK;
}

static inline uint64_t to_physical(const std::vector<int>& perm, uint64_t logical)
{
    uint64_t p = 0;
    for (size_t q = 0; q < perm.size(); q++)
        if ((logical >> q) & 1) p |= 1ull << perm[q];
    return p;
}

template <typename R>
int amplitudes(sv_state* s, const uint64_t* idx, size_t m, double* out)
{
    const uint64_t dim = 1ull << s->n;
    for (size_t i = 0; i < m; i++)
        if (idx[i] >= dim) return fail(s, SV_ERR_ARG, "amplitude index out of range");
    if (m == 0) return SV_OK;
    const size_t batch = std::min<size_t>(m, (size_t)1 << 22);
    uint64_t *d_loc = nullptr, *d_dst = nullptr;
    double* d_out = nullptr;
    cudaError_t e;
    int r = SV_OK;
    if ((e = dev_alloc(s, &d_loc, batch * 8)) || (e = dev_alloc(s, &d_dst, batch * 8)) ||
        (e = dev_alloc(s, &d_out, batch * 16))) {
        dev_free(s, d_loc); dev_free(s, d_dst); dev_free(s, d_out);
        return cuda_fail(s, e, "cudaMalloc(gather)");
    }
    std::vector<uint64_t> loc, dst;
    for (size_t b0 = 0; b0 < m && !r; b0 += batch) {
        const size_t nb = std::min(batch, m - b0);
        if (s->mode == SV_UNCOMPRESSED) {
            loc.resize(nb);
            dst.resize(nb);
            for (size_t i = 0; i < nb; i++) { loc[i] = to_physical(s->perm, idx[b0 + i]); dst[i] = i; }
            if ((e = cudaMemcpyAsync(d_loc, loc.data(), nb * 8, cudaMemcpyHostToDevice, s->s_comp)) ||
                (e = cudaMemcpyAsync(d_dst, dst.data(), nb * 8, cudaMemcpyHostToDevice, s->s_comp)) ||
                (e = launch_gather<R>(s->d_state, d_loc, d_dst, nb, d_out, s->s_comp))) {
                r = cuda_fail(s, e, "gather");
                break;
            }
            s->st.kernel_launches++;
        } else {
            // bucket requests by chunk
            std::vector<std::pair<uint64_t, uint64_t>> req(nb);  // (physical, position)
            for (size_t i = 0; i < nb; i++) req[i] = {to_physical(s->perm, idx[b0 + i]), i};
            std::sort(req.begin(), req.end());
            const int gcap = 1 << std::min(s->gmax, s->nh);
            size_t i = 0;
            while (i < nb && !r) {
                std::vector<uint64_t> ks;
                loc.clear();
                dst.clear();
                while (i < nb) {
                    const uint64_t k = req[i].first >> s->c;
                    if (ks.empty() || ks.back() != k) {
                        if ((int)ks.size() == gcap) break;
                        ks.push_back(k);
                    }
                    loc.push_back(((uint64_t)(ks.size() - 1) << s->c) | (req[i].first & ((1ull << s->c) - 1)));
                    dst.push_back(req[i].second);
                    i++;
                }
                if ((r = stage_chunks<R>(s, ks))) break;
                if ((e = cudaMemcpyAsync(d_loc, loc.data(), loc.size() * 8, cudaMemcpyHostToDevice, s->s_comp)) ||
                    (e = cudaMemcpyAsync(d_dst, dst.data(), dst.size() * 8, cudaMemcpyHostToDevice, s->s_comp)) ||
                    (e = launch_gather<R>(s->d_amps, d_loc, d_dst, loc.size(), d_out, s->s_comp))) {
                    r = cuda_fail(s, e, "gather");
                    break;
                }
                s->st.kernel_launches++;
                // loc/dst are host vectors reused next round: wait before overwriting them
                if ((r = wait_stream(s, s->s_comp))) break;
            }
        }
        if (r) break;
        if ((e = cudaMemcpyAsync(out + 2 * b0, d_out, nb * 16, cudaMemcpyDeviceToHost, s->s_comp))) {
            r = cuda_fail(s, e, "D2H amplitudes");
            break;
        }
        r = wait_stream(s, s->s_comp);
    }
    if (!r) r = check_device_error(s);
    dev_free(s, d_loc);
    dev_free(s, d_dst);
    dev_free(s, d_out);
    return r;
}

// -------------------------------------------------------------- overlap
// <a|b> in FP64 with b held whole in HBM: a's amplitudes are read where they
// are (a's state in HBM, or its chunks staged and decoded group by group) and
// paired with b's amplitude of the same logical index through the two
// states' qubit maps.
template <typename RA, typename RB>
int inner(sv_state* a, const sv_state* b, double* out)
{
    IndexMap map;
    map.n = a->n;
    for (int q = 0; q < a->n; q++) {
        map.pos[a->perm[q]] = (int8_t)b->perm[q];
        if (a->perm[q] != b->perm[q]) map.identity = 0;
    }
    const uint64_t run = a->mode == SV_UNCOMPRESSED ? (1ull << a->n) : (1ull << (a->c + std::min(a->gmax, a->nh)));
    const int nb = reduce_blocks_for(run);
    double* d_part = nullptr;
    double* d_out = nullptr;
    cudaError_t e;
    if ((e = dev_alloc(a, &d_part, sizeof(double) * 2 * nb)) || (e = dev_alloc(a, &d_out, sizeof(double) * 2))) {
        dev_free(a, d_part);
        dev_free(a, d_out);
        return cuda_fail(a, e, "cudaMalloc(inner)");
    }
    int r = SV_OK;
    if ((e = cudaMemsetAsync(d_out, 0, sizeof(double) * 2, a->s_comp))) r = cuda_fail(a, e, "memset");
    if (!r && a->mode == SV_UNCOMPRESSED) {
        if ((e = launch_inner<RA, RB>(a->d_state, run, 0, b->d_state, map, d_part, nb, a->s_comp)) ||
            (e = launch_sum_partials(d_part, 2, nb, d_out, a->s_comp)))
            r = cuda_fail(a, e, "inner");
        a->st.kernel_launches += 2;
    } else if (!r) {
        const uint64_t nch = 1ull << a->nh, gcap = 1ull << std::min(a->gmax, a->nh);
        std::vector<uint64_t> ks;
        for (uint64_t k0 = 0; k0 < nch && !r; k0 += gcap) {
            ks.clear();
            for (uint64_t k = k0; k < k0 + gcap; k++) ks.push_back(k);
            if ((r = stage_chunks<RA>(a, ks))) break;
            if ((e = launch_inner<RA, RB>(a->d_amps, gcap << a->c, k0 << a->c, b->d_state, map, d_part, nb,
                                          a->s_comp)) ||
                (e = launch_sum_partials(d_part, 2, nb, d_out, a->s_comp)))
                r = cuda_fail(a, e, "inner");
            a->st.kernel_launches += 2;
        }
    }
    if (!r && (e = cudaMemcpyAsync(out, d_out, sizeof(double) * 2, cudaMemcpyDeviceToHost, a->s_comp)))
        r = cuda_fail(a, e, "D2H inner");
    if (!r) r = wait_stream(a, a->s_comp);
    if (!r) r = check_device_error(a);
    dev_free(a, d_part);
    dev_free(a, d_out);
    return r;
}

// ------------------------------------------------------------ expectation
static PauliDev pauli_dev(const sv_pauli_term& t, uint64_t xl, uint64_t zl, uint64_t zg, double scale)
{
    PauliDev p{};
    p.coeff = t.coeff * scale;
    p.xl = xl;
    p.zl = zl;
    p.zg = zg;
    p.ny = __builtin_popcountll(t.xmask & t.zmask) & 3;
    return p;
}

static uint64_t mask_to_physical(const std::vector<int>& perm, uint64_t m) { return to_physical(perm, m); }

// <psi| sum_t c_t P_t |psi> term group by term group: per distinct high
// x-mask, chunk pairs (k, k ^ x) staged together (any x; the path for masks
// wider than a staging group and for term counts beyond the one-sweep kernel).
template <typename R>
static int expect_pairs(sv_state* s, const std::vector<sv_pauli_term>& phys, double* out_re)
{
    *out_re = 0;
    const size_t nterms = phys.size();
    if (nterms == 0) return SV_OK;
    cudaError_t e;
    const int c = s->mode == SV_UNCOMPRESSED ? s->n : s->c;
    const uint64_t lowmask = (c >= 64) ? ~0ull : ((1ull << c) - 1);
    const int nblocks = reduce_blocks_for(1ull << c);
    // group by the high part of x
    std::vector<uint64_t> xhs;
    for (auto& t : phys) xhs.push_back(t.xmask >> c);
    std::sort(xhs.begin(), xhs.end());
    xhs.erase(std::unique(xhs.begin(), xhs.end()), xhs.end());
    PauliDev* d_terms = nullptr;
    double *d_part = nullptr, *d_acc = nullptr;
    if ((e = dev_alloc(s, &d_terms, sizeof(PauliDev) * nterms)) ||
        (e = dev_alloc(s, &d_part, sizeof(double) * nterms * nblocks)) || (e = dev_alloc(s, &d_acc, sizeof(double) * nterms))) {
        dev_free(s, d_terms); dev_free(s, d_part); dev_free(s, d_acc);
        return cuda_fail(s, e, "cudaMalloc(expect)");
    }
    int r = SV_OK;
    cudaMemsetAsync(d_acc, 0, sizeof(double) * nterms, s->s_comp);
    std::vector<PauliDev> hd;
    size_t acc_off = 0;
    std::vector<std::pair<size_t, size_t>> acc_map;  // (term index, slot in d_acc)
    for (uint64_t xh : xhs) {
        hd.clear();
        std::vector<size_t> tid;
        const double pair_scale = xh ? 2.0 : 1.0;
        for (size_t i = 0; i < nterms; i++) {
            if ((phys[i].xmask >> c) != xh) continue;
            hd.push_back(pauli_dev(phys[i], phys[i].xmask & lowmask, phys[i].zmask & lowmask, phys[i].zmask & ~lowmask,
                                   pair_scale));
            tid.push_back(i);
        }
        const int nt = (int)hd.size();
        if ((e = cudaMemcpyAsync(d_terms, hd.data(), sizeof(PauliDev) * nt, cudaMemcpyHostToDevice, s->s_comp))) {
            r = cuda_fail(s, e, "upload terms");
            break;
        }
        if (s->mode == SV_UNCOMPRESSED) {
            if ((e = launch_pauli_partials<R>(s->d_state, s->d_state, s->n, 0, d_terms, nt, d_part, nblocks, s->s_comp)) ||
                (e = launch_sum_partials(d_part, nt, nblocks, d_acc + acc_off, s->s_comp))) {
                r = cuda_fail(s, e, "pauli");
                break;
            }
            s->st.kernel_launches += 2;
        } else {
            // units: chunk k (xh == 0) or pairs (k, k ^ xh) with k < k ^ xh
            const uint64_t nch = 1ull << s->nh;
            std::vector<uint64_t> units;
            for (uint64_t k = 0; k < nch; k++)
                if (xh == 0 || k < (k ^ xh)) units.push_back(k);
            const size_t per = xh ? (size_t)(1 << (s->gmax - 1)) : (size_t)(1 << s->gmax);
            for (size_t u0 = 0; u0 < units.size() && !r; u0 += per) {
                const size_t nu = std::min(per, units.size() - u0);
                std::vector<uint64_t> ks;
                for (size_t u = 0; u < nu; u++) {
                    ks.push_back(units[u0 + u]);
                    if (xh) ks.push_back(units[u0 + u] ^ xh);
                }
                if ((r = stage_chunks<R>(s, ks))) break;
                const size_t cb = sizeof(R) * 2ull << s->c;
                for (size_t u = 0; u < nu; u++) {
                    const uint8_t* A = static_cast<const uint8_t*>(s->d_amps) + (xh ? 2 * u : u) * cb;
                    const uint8_t* B = xh ? A + cb : A;
                    if ((e = launch_pauli_partials<R>(A, B, s->c, units[u0 + u] << s->c, d_terms, nt, d_part, nblocks,
                                                      s->s_comp)) ||
                        (e = launch_sum_partials(d_part, nt, nblocks, d_acc + acc_off, s->s_comp))) {
                        r = cuda_fail(s, e, "pauli");
                        break;
                    }
                    s->st.kernel_launches += 2;
                }
            }
            if (r) break;
        }
        for (int j = 0; j < nt; j++) acc_map.push_back({tid[j], acc_off + j});
        acc_off += nt;
        // hd is reused next round: the upload above is stream-ordered before the next upload
    }
    if (!r) {
        std::vector<double> acc(nterms);
        if ((e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * nterms, cudaMemcpyDeviceToHost, s->s_comp)))
            r = cuda_fail(s, e, "D2H expect");
        else if (!(r = wait_stream(s, s->s_comp))) {
            std::vector<double> per_term(nterms, 0.0);
            for (auto& pm : acc_map) per_term[pm.first] = acc[pm.second];
            double sum = 0;
            for (size_t i = 0; i < nterms; i++) sum += per_term[i];
            *out_re = sum;
        }
    }
    if (!r) r = check_device_error(s);
    dev_free(s, d_terms);
    dev_free(s, d_part);
    dev_free(s, d_acc);
    return r;
}

// <psi|H|psi> of the compressed store in few streaming sweeps: a sweep with
// staged high qubits S decodes each chunk group as a local state of c + |S|
// qubits (S[j] at local bit c + j), on which every term whose high x-mask
// lies in S is evaluated by one all-terms kernel; the z-mask on the group's
// fixed high bits is a sign per group. The staged sets are chosen greedily
// to cover the distinct high x-masks (the Ising chain: two sweeps). Chunk
// copies to the device alternate between two stream slots so that the next
// group's copies overlap this group's decode and reduction.
// The terms of one sweep over a 2^L buffer, grouped for k_energy_tiles: each
// set's terms have x-masks whose bits above local bit 7 fit the set's four
// tile positions, so their partners are read from the tile in shared
// memory; the rest (more than four such bits, or buffers under 2^12
// amplitudes) go to k_energy. hd is reordered: the sets' terms first,
// contiguous, then the rest.
struct EnergyPlan {
    std::vector<EnergyTiles> tiles;
    std::vector<int> off, cnt;
    int rest_off = 0, rest_cnt = 0;
};

static EnergyPlan energy_plan(std::vector<PauliDev>& hd, int L)
{
    EnergyPlan ep;
    const int nt = (int)hd.size();
    std::vector<int> rest, order(nt);
    std::vector<uint64_t> H;                   // each set's tile positions above bit 7
    std::vector<std::vector<int>> members;
    for (int i = 0; i < nt; i++) order[i] = i;
    if (L >= kEnergyTileBits) {
        auto need = [&](int i) { return hd[i].xl & ~0xFFull; };
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return __builtin_popcountll(need(a)) > __builtin_popcountll(need(b)); });
        std::vector<int> free_terms;
        for (int i : order) {
            const uint64_t nd = need(i);
            if (__builtin_popcountll(nd) > 4) {
                rest.push_back(i);
                continue;
            }
            if (!nd) {
                free_terms.push_back(i);
                continue;
            }
            int best = -1, best_ov = -1;
            for (size_t k = 0; k < H.size(); k++) {
                if (__builtin_popcountll(H[k] | nd) > 4) continue;
                const int ov = __builtin_popcountll(H[k] & nd);
                if (ov > best_ov) {
                    best = (int)k;
                    best_ov = ov;
                }
            }
            if (best < 0) {
                H.push_back(nd);
                members.push_back({i});
            } else {
                H[best] |= nd;
                members[best].push_back(i);
            }
        }
        if (!free_terms.empty()) {
            if (H.empty()) {
                H.push_back(0);
                members.push_back({});
            }
            for (int i : free_terms) members[0].push_back(i);
        }
    } else {
        rest = order;
    }
    std::vector<PauliDev> out;
    for (size_t k = 0; k < H.size(); k++) {
        uint64_t h = H[k];
        for (int p = 8; p < L && __builtin_popcountll(h) < 4; p++) h |= 1ull << p;
        EnergyTiles et{};
        int j = 0, o = 0;
        for (int p = 0; p < L; p++) {
            if ((h >> p) & 1) et.hp[j++] = (int8_t)p;
            else if (p >= 8) et.op[o++] = (int8_t)p;
        }
        et.nout = o;
        ep.tiles.push_back(et);
        ep.off.push_back((int)out.size());
        for (int i : members[k]) out.push_back(hd[i]);
        ep.cnt.push_back((int)out.size() - ep.off.back());
    }
    ep.rest_off = (int)out.size();
    for (int i : rest) out.push_back(hd[i]);
    ep.rest_cnt = (int)out.size() - ep.rest_off;
    hd.swap(out);
    return ep;
}

// <psi|H|psi> partial sums of a 2^L buffer added to *d_acc on stream st.
template <typename R>
static cudaError_t energy_sweep(sv_state* s, const void* psi, int L, uint64_t gbase, const EnergyPlan& ep,
                                const PauliDev* d_terms, double* d_part, int nblocks, double* d_acc)
{
    cudaError_t e;
    for (size_t k = 0; k < ep.tiles.size(); k++) {
        if (!ep.cnt[k]) continue;
        if ((e = launch_energy_tiles<R>(psi, L, gbase, ep.tiles[k], d_terms + ep.off[k], ep.cnt[k], d_part, nblocks,
                                        s->d_err, s->s_comp)) ||
            (e = launch_sum_partials(d_part, 1, nblocks, d_acc, s->s_comp)))
            return e;
        s->st.kernel_launches += 2;
    }
    if (ep.rest_cnt) {
        if ((e = launch_energy_partials<R>(psi, L, gbase, d_terms + ep.rest_off, ep.rest_cnt, d_part, nblocks,
                                           s->s_comp)) ||
            (e = launch_sum_partials(d_part, 1, nblocks, d_acc, s->s_comp)))
            return e;
        s->st.kernel_launches += 2;
    }
    return cudaSuccess;
}

template <typename R>
static int expect_streamed(sv_state* s, const std::vector<sv_pauli_term>& phys, double* out_re)
{
    *out_re = 0;
    const int c = s->c, nh = s->nh, g = std::min(s->gmax, nh);
    const uint64_t lowmask = (1ull << c) - 1;
    std::vector<sv_pauli_term> wide;
    std::vector<size_t> sweepable;
    for (size_t i = 0; i < phys.size(); i++) {
        if (__builtin_popcountll(phys[i].xmask >> c) > g) wide.push_back(phys[i]);
        else sweepable.push_back(i);
    }
    // staged sets (bit masks over the nh chunk-index bits), each with its terms
    std::vector<std::pair<uint64_t, std::vector<size_t>>> sweeps;
    std::vector<size_t> todo = sweepable;
    std::stable_sort(todo.begin(), todo.end(), [&](size_t a, size_t b) {
        return __builtin_popcountll(phys[a].xmask >> c) > __builtin_popcountll(phys[b].xmask >> c);
    });
    while (!todo.empty()) {
        uint64_t S = 0;
        for (size_t i : todo) {
            const uint64_t m = phys[i].xmask >> c;
            if (__builtin_popcountll(S | m) <= g) S |= m;
        }
        for (int b = 0; b < nh && __builtin_popcountll(S) < g; b++) S |= 1ull << b;
        std::vector<size_t> mine, rest;
        for (size_t i : todo) ((((phys[i].xmask >> c) & ~S) == 0) ? mine : rest).push_back(i);
        sweeps.push_back({S, mine});
        todo.swap(rest);
    }
    const int nblocks = reduce_blocks_for(1ull << (c + g));
    PauliDev* d_terms = nullptr;
    double *d_part = nullptr, *d_acc = nullptr;
    cudaError_t e;
    if ((e = dev_alloc(s, &d_terms, sizeof(PauliDev) * std::max<size_t>(1, phys.size()))) ||
        (e = dev_alloc(s, &d_part, sizeof(double) * nblocks)) || (e = dev_alloc(s, &d_acc, sizeof(double)))) {
        dev_free(s, d_terms); dev_free(s, d_part); dev_free(s, d_acc);
        return cuda_fail(s, e, "cudaMalloc(expect)");
    }
    int r = SV_OK;
    if ((e = cudaMemsetAsync(d_acc, 0, sizeof(double), s->s_comp))) r = cuda_fail(s, e, "memset");
    uint64_t issued = 0;  // groups issued so far (stream slot = issued & 1)
    for (size_t sw = 0; sw < sweeps.size() && !r; sw++) {
        const uint64_t S = sweeps[sw].first;
        std::vector<int> spos, fpos;
        for (int b = 0; b < nh; b++) (((S >> b) & 1) ? spos : fpos).push_back(b);
        std::vector<PauliDev> hd;
        for (size_t i : sweeps[sw].second) {
            const sv_pauli_term& t = phys[i];
            const uint64_t xh = t.xmask >> c, zh = t.zmask >> c;
            uint64_t xl = t.xmask & lowmask, zl = t.zmask & lowmask;
            for (size_t j = 0; j < spos.size(); j++) {
                xl |= ((xh >> spos[j]) & 1ull) << (c + j);
                zl |= ((zh >> spos[j]) & 1ull) << (c + j);
            }
            hd.push_back(pauli_dev(t, xl, zl, t.zmask & ~lowmask & ~(S << c), 1.0));
        }
        const EnergyPlan ep = energy_plan(hd, c + g);
        // the previous sweep's reductions read d_terms: the upload waits for them
        if ((e = cudaMemcpyAsync(d_terms, hd.data(), sizeof(PauliDev) * hd.size(), cudaMemcpyHostToDevice, s->s_comp)) ||
            (e = cudaStreamSynchronize(s->s_comp))) {
            r = cuda_fail(s, e, "upload terms");
            break;
        }
        const int gch = 1 << g;
        const uint64_t ngroups = 1ull << fpos.size();
        for (uint64_t gi = 0; gi < ngroups && !r; gi++, issued++) {
            const int slot = (int)(issued & 1);
            const uint64_t base = deposit(gi, fpos);
            // the slot's streams are overwritten once its previous decode is done
            if (issued >= 2 && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_h2d[2 + slot], 0))) {
                r = cuda_fail(s, e, "wait decode");
                break;
            }
            GroupIn gin{};
            for (int j = 0; j < gch && !r; j++) {
                const ChunkRef& cr = s->cur[base | deposit((uint64_t)j, spos)];
                gin.bytes[j] = (uint32_t)cr.bytes;
                if ((e = cudaMemcpyAsync(s->d_in[slot] + (size_t)j * s->stride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice,
                                         s->s_h2d)))
                    r = cuda_fail(s, e, "H2D chunk");
                s->st.bytes_h2d += cr.bytes;
            }
            if (r) break;
            if ((e = cudaEventRecord(s->ev_h2d[slot], s->s_h2d)) ||
                (e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[slot], 0)) ||
                (e = launch_decode<R>(s->d_in[slot], s->stride, c, s->dtype, gch, gin, s->d_amps, s->scale, s->d_err,
                                      s->s_comp)) ||
                (e = cudaEventRecord(s->ev_h2d[2 + slot], s->s_comp)) ||
                (e = energy_sweep<R>(s, s->d_amps, c + g, base << c, ep, d_terms, d_part, nblocks, d_acc))) {
                r = cuda_fail(s, e, "expect group");
                break;
            }
            s->st.kernel_launches += 1;
        }
    }
    double acc = 0;
    const int rs = sync_all(s);
    if (!r && !rs && (e = cudaMemcpy(&acc, d_acc, sizeof(double), cudaMemcpyDeviceToHost))) r = cuda_fail(s, e, "D2H expect");
    dev_free(s, d_terms);
    dev_free(s, d_part);
    dev_free(s, d_acc);
    if (r || rs) return r ? r : rs;
    double rest = 0;
    if (!wide.empty() && (r = expect_pairs<R>(s, wide, &rest))) return r;
    *out_re = acc + rest;
    return check_device_error(s);
}

template <typename R>
int expect(sv_state* s, const sv_pauli_term* terms, size_t nterms, double* out_re)
{
    *out_re = 0;
    if (nterms == 0) return SV_OK;
    const uint64_t dim_mask = (s->n >= 64) ? ~0ull : ((1ull << s->n) - 1);
    for (size_t i = 0; i < nterms; i++)
        if ((terms[i].xmask | terms[i].zmask) & ~dim_mask) return fail(s, SV_ERR_ARG, "Pauli mask out of range");
    // physical masks
    std::vector<sv_pauli_term> phys(nterms);
    for (size_t i = 0; i < nterms; i++) {
        phys[i] = terms[i];
        phys[i].xmask = mask_to_physical(s->perm, terms[i].xmask);
        phys[i].zmask = mask_to_physical(s->perm, terms[i].zmask);
    }
    if ((int)nterms > max_energy_terms()) return expect_pairs<R>(s, phys, out_re);
    if (s->mode == SV_COMPRESSED) return expect_streamed<R>(s, phys, out_re);
    // whole state in HBM: every term in one sweep
    const int nblocks = reduce_blocks_for(1ull << s->n);
    std::vector<PauliDev> hd;
    for (const auto& t : phys) hd.push_back(pauli_dev(t, t.xmask, t.zmask, 0, 1.0));
    const EnergyPlan ep = energy_plan(hd, s->n);
    PauliDev* d_terms = nullptr;
    double *d_part = nullptr, *d_acc = nullptr;
    cudaError_t e;
    if ((e = dev_alloc(s, &d_terms, sizeof(PauliDev) * nterms)) || (e = dev_alloc(s, &d_part, sizeof(double) * nblocks)) ||
        (e = dev_alloc(s, &d_acc, sizeof(double)))) {
        dev_free(s, d_terms); dev_free(s, d_part); dev_free(s, d_acc);
        return cuda_fail(s, e, "cudaMalloc(expect)");
    }
    int r = SV_OK;
    double acc = 0;
    if ((e = cudaMemcpyAsync(d_terms, hd.data(), sizeof(PauliDev) * nterms, cudaMemcpyHostToDevice, s->s_comp)) ||
        (e = cudaMemsetAsync(d_acc, 0, sizeof(double), s->s_comp)) ||
        (e = energy_sweep<R>(s, s->d_state, s->n, 0, ep, d_terms, d_part, nblocks, d_acc)) ||
        (e = cudaMemcpyAsync(&acc, d_acc, sizeof(double), cudaMemcpyDeviceToHost, s->s_comp)))
        r = cuda_fail(s, e, "energy");
    if (!r) r = wait_stream(s, s->s_comp);
    dev_free(s, d_terms);
    dev_free(s, d_part);
    dev_free(s, d_acc);
    if (r) return r;
    *out_re = acc;
    return check_device_error(s);
}

// --------------------------------------------------------------- adjoint
template <typename R>
int grad_uncompressed(sv_state* s, const std::vector<PGate>& gates, size_t nparams, const sv_pauli_term* H,
                      size_t nterms, double* energy, double* grad)
{
    cudaError_t e;
    const int n = s->n;
    const size_t vbytes = sizeof(R) * 2ull << n;
    if (!s->d_lam) {
        if ((e = dev_alloc(s, &s->d_lam, vbytes))) return cuda_fail(s, e, "cudaMalloc(lambda)");
    }
    int r = init_state<R>(s);
    if (r) return r;
    std::vector<int> ids(gates.size());
    for (size_t i = 0; i < gates.size(); i++) ids[i] = (int)i;
    if ((r = run_pass_uncompressed<R>(s, s->d_state, gates, ids))) return r;
    // lambda = H psi (physical masks)
    std::vector<PauliDev> hd;
    for (size_t i = 0; i < nterms; i++) {
        sv_pauli_term t = H[i];
        const uint64_t x = mask_to_physical(s->perm, t.xmask), z = mask_to_physical(s->perm, t.zmask);
        hd.push_back(pauli_dev(t, x, z, 0, 1.0));
    }
    PauliDev* d_terms = nullptr;
    double *d_part = nullptr, *d_acc = nullptr, *d_gpart = nullptr;
    const int nblocks = reduce_blocks_for(1ull << n);
    // reverse sweep plan
    std::vector<int> rids(gates.size());
    for (size_t i = 0; i < gates.size(); i++) rids[i] = (int)(gates.size() - 1 - i);
    std::vector<PGate> inv(gates.size());
    for (size_t i = 0; i < gates.size(); i++) {
        inv[i] = gates[i];
        const int K = 1 << gates[i].nt;
        for (int a = 0; a < K; a++)
            for (int b = 0; b < K; b++) inv[i].m[a * K + b] = std::conj(gates[i].m[b * K + a]);
    }
    const int L = n;
    int t, l;
    tile_shape(L, std::min(s->tq, 12), s->lq, t, l);
    const std::vector<int> noS;
    const std::vector<HOp> hops = local_ops(inv, rids, L, noS, true);
    const std::vector<SubPlan> subs = plan_subpasses(hops, L, t, l, true);
    std::vector<TileDesc> tds;
    std::vector<int> offs, cnts, slot_params;
    std::vector<DevOp<R>> ops;
    std::vector<int> slot_base;
    int max_slots = 0;
    AdjPlan<R> ap;
    if ((r = jit_adjoint_plan<R>(s, subs, L, t, l, slot_params, ap))) return r;
    if (ap.ok) {
        tds = ap.td;
        slot_base = ap.gslot;
        for (int v : ap.nsl) max_slots = std::max(max_slots, v);
    } else {
        for (const SubPlan& sp : subs) {
            TileDesc td = tile_desc(sp.T, L, t, l);
            tds.push_back(td);
            offs.push_back((int)ops.size());
            slot_base.push_back((int)slot_params.size());
            int base = 0;
            dev_ops<R>(sp, td, ops, &base, &slot_params);
            max_slots = std::max(max_slots, base);
            cnts.push_back((int)ops.size() - offs.back());
        }
    }
    const uint64_t ntiles = 1ull << (L - t);
    const size_t nslots_total = slot_params.size();
    if ((e = dev_alloc(s, &d_terms, sizeof(PauliDev) * std::max<size_t>(1, nterms))) ||
        (e = dev_alloc(s, &d_part, sizeof(double) * nblocks)) ||
        (e = dev_alloc(s, &d_acc, sizeof(double) * (1 + std::max<size_t>(1, nslots_total)))) ||
        (e = dev_alloc(s, &d_gpart, sizeof(double) * std::max(1, max_slots) * ntiles))) {
        dev_free(s, d_terms); dev_free(s, d_part); dev_free(s, d_acc); dev_free(s, d_gpart);
        return cuda_fail(s, e, "cudaMalloc(grad)");
    }
    do {
        if (nterms &&
            (e = cudaMemcpyAsync(d_terms, hd.data(), sizeof(PauliDev) * nterms, cudaMemcpyHostToDevice, s->s_comp))) {
            r = cuda_fail(s, e, "upload H");
            break;
        }
        if ((e = launch_hamiltonian<R>(s->d_state, s->d_lam, n, d_terms, (int)nterms, s->s_comp))) {
            r = cuda_fail(s, e, "hamiltonian");
            break;
        }
        cudaMemsetAsync(d_acc, 0, sizeof(double) * (1 + nslots_total), s->s_comp);
        if ((e = launch_dot<R>(s->d_state, s->d_lam, 1ull << n, d_part, nblocks, s->s_comp)) ||
            (e = launch_sum_partials(d_part, 1, nblocks, d_acc, s->s_comp))) {
            r = cuda_fail(s, e, "energy");
            break;
        }
        s->st.kernel_launches += 3;
        if (!ap.ok && (r = upload_ops<R>(s, ops))) break;
        const DevOp<R>* d_ops = static_cast<const DevOp<R>*>(s->d_ops);
        for (size_t i = 0; i < tds.size(); i++) {
            unsigned parts = (unsigned)ntiles;  // gradient partials per slot
            if (ap.ok) {
                e = jit_launch_adjoint<R>(ap.fn[i], s->d_state, s->d_lam, tds[i], 0, d_gpart, ap.par[i], s->s_comp,
                                          &parts);
                s->st.jit_launches++;
                s->st.jit_adjoint_launches++;
            } else {
                e = launch_adjoint<R>(s->d_state, s->d_lam, tds[i], d_ops + offs[i], cnts[i], 0, d_gpart, ntiles,
                                      s->s_comp);
            }
            if (e) {
                r = cuda_fail(s, e, "adjoint");
                break;
            }
            s->st.kernel_launches++;
            const int nsl = (i + 1 < tds.size() ? slot_base[i + 1] : (int)nslots_total) - slot_base[i];
            if (nsl > 0) {
                if ((e = launch_sum_partials(d_gpart, nsl, (int)parts, d_acc + 1 + slot_base[i], s->s_comp))) {
                    r = cuda_fail(s, e, "grad reduce");
                    break;
                }
                s->st.kernel_launches++;
            }
        }
        if (r) break;
        s->st.subpasses += tds.size();
        std::vector<double> acc(1 + nslots_total);
        if ((e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, s->s_comp))) {
            r = cuda_fail(s, e, "D2H grad");
            break;
        }
        if ((r = wait_stream(s, s->s_comp))) break;
        *energy = acc[0];
        for (size_t p = 0; p < nparams; p++) grad[p] = 0;
        for (size_t j = 0; j < nslots_total; j++) grad[slot_params[j]] += acc[1 + j];
    } while (0);
    dev_free(s, d_terms);
    dev_free(s, d_part);
    dev_free(s, d_acc);
    dev_free(s, d_gpart);
    if (!r) r = check_device_error(s);
    return r;
}

// ----------------------------------------------------- compressed adjoint
// Adjoint gradient with psi and lambda = H psi both held as compressed chunk
// stores in pinned host memory. The reverse sweep runs the forward plan's
// passes in reverse order, each pass's gates reversed and daggered, streaming
// the chunk groups of both vectors through the GPU.
template <typename R>
static int ensure_lambda_store(sv_state* s)
{
    if (s->d_amps2) return SV_OK;
    const int gsz = std::min(s->gmax, s->nh);
    const uint64_t gch = 1ull << gsz;
    cudaError_t e;
    if ((e = dev_alloc(s, &s->d_amps2, ((sizeof(R) * 2) << s->c) * gch))) {
        cudaGetLastError();
        return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the lambda group buffer failed");
    }
    for (int i = 0; i < s->nslots; i++) {
        if ((e = dev_alloc(s, &s->d_in2[i], s->stride * gch)) || (e = dev_alloc(s, &s->d_out2[i], s->stride * gch)) ||
            (e = dev_alloc(s, &s->d_co2[i], sizeof(ChunkOut) * gch))) {
            cudaGetLastError();
            return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the lambda staging slots failed");
        }
        if ((e = cudaHostAlloc(&s->h_co2[i], sizeof(ChunkOut) * gch, cudaHostAllocDefault)))
            return fail(s, SV_ERR_HOST_OOM, "pinned allocation failed");
    }
    const uint64_t nchunks = 1ull << s->nh;
    s->lcur.assign(nchunks, ChunkRef{});
    s->lpool.seg_bytes = s->pool.seg_bytes;
    return SV_OK;
}

// lambda = H psi, one output chunk at a time from the staged source chunks
// k ^ xh (one per distinct high x-mask); adds Re<psi_k|lambda_k> to *d_energy.
// When the distinct high x-masks outnumber the chunks a staging group holds,
// they are taken in batches: every batch stages chunk k itself in slot 0 and
// as many other sources as fit, and lambda_k accumulates over the batches in
// device memory before it is encoded once. With a single batch that fits
// twice, two staging sets alternate: chunk k+1's sources cross the host link
// while chunk k is decoded, multiplied and encoded, and chunk k's stream
// returns to the host while chunk k+1 computes. With lambda_cache 1 and room
// on the device for the whole decoded psi, psi is instead decoded once and
// each output chunk reads its sources there, and its output staging sets
// alternate the same way. d_terms holds every batch's term table for every
// output chunk (2^(n-c) x phys.size() entries).
template <typename R>
static int build_lambda(sv_state* s, const std::vector<sv_pauli_term>& phys, PauliDev* d_terms, double* d_part,
                        int nblocks, double* d_energy)
{
    const int c = s->c;
    const uint64_t lowmask = (1ull << c) - 1;
    std::vector<uint64_t> X{0};
    for (const auto& t : phys) X.push_back(t.xmask >> c);
    std::sort(X.begin(), X.end());
    X.erase(std::unique(X.begin(), X.end()), X.end());  // X[0] = 0: chunk k itself
    const size_t gcap = (size_t)1 << std::min(s->gmax, s->nh);
    if (gcap < 2 && X.size() > 1) return fail(s, SV_ERR_ARG, "staging groups too small for lambda = H psi");
    const uint64_t nch = 1ull << s->nh;
    const size_t amp_bytes = sizeof(R) * 2;
    cudaError_t e;
    // lambda_cache 1: when the whole decoded psi fits in half the free device
    // memory (or the caller's allocator grants it), psi is decoded into it
    // once and every output chunk reads its sources there (ψ decoded once
    // instead of once per source); a term's slot is then its source chunk.
    void* d_full = nullptr;
    if (s->cfg.lambda_cache == 1 && X.size() > 1) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        cudaGetLastError();
        const size_t full_bytes = amp_bytes << s->n;
        if ((s->cfg.device_alloc || (double)full_bytes <= 0.5 * (double)free_b) && dev_alloc(s, &d_full, full_bytes)) {
            cudaGetLastError();
            d_full = nullptr;
        }
    }
    struct FullFree {
        sv_state* s;
        void*& p;
        ~FullFree()
        {
            if (p) {
                cudaStreamSynchronize(s->s_comp);  // the kernels that read it
                dev_free(s, p);
            }
        }
    } full_free{s, d_full};
    // batches of source slots: batch 0 = X[0 .. gcap), later ones X[0] and the
    // next gcap - 1; one batch of every source when psi is decoded in full
    std::vector<std::vector<size_t>> batch{{}};
    for (size_t j = 0; j < X.size(); j++) {
        if (!d_full && batch.back().size() == gcap) batch.push_back({0});
        batch.back().push_back(j);
    }
    const size_t nb = batch.size(), nt = phys.size();
    std::vector<int> batch_of(X.size(), -1), slot_of(X.size(), -1);
    for (size_t b = 0; b < nb; b++)
        for (size_t i = 0; i < batch[b].size(); i++)
            if (batch_of[batch[b][i]] < 0) {
                batch_of[batch[b][i]] = (int)b;
                slot_of[batch[b][i]] = (int)i;
            }
    const size_t m = batch[0].size();
    const int nset = (d_full || (nb == 1 && 2 * m <= gcap)) ? 2 : 1;
    // term table of (chunk k, batch b) at d_terms + toff[b] + k * tcnt[b]
    std::vector<size_t> toff(nb, 0), tcnt(nb, 0);
    for (size_t i = 0; i < nt; i++) {
        const size_t j = std::lower_bound(X.begin(), X.end(), phys[i].xmask >> c) - X.begin();
        tcnt[batch_of[j]]++;
    }
    for (size_t b = 1; b < nb; b++) toff[b] = toff[b - 1] + nch * tcnt[b - 1];
    if (nt) {
        // each table lists the terms that read one source (slot, low x-mask)
        // together: the kernel loads a source once per run of such terms
        std::vector<size_t> ord(nt);
        for (size_t i = 0; i < nt; i++) ord[i] = i;
        auto slot_key = [&](size_t i) {
            const size_t j = std::lower_bound(X.begin(), X.end(), phys[i].xmask >> c) - X.begin();
            return std::make_pair(slot_of[j], phys[i].xmask & lowmask);
        };
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return slot_key(a) < slot_key(b); });
        std::vector<PauliDev> hd(nch * nt);
        for (uint64_t k = 0; k < nch; k++) {
            std::vector<size_t> fill(nb, 0);
            for (size_t i : ord) {
                const uint64_t xh = phys[i].xmask >> c;
                const size_t j = std::lower_bound(X.begin(), X.end(), xh) - X.begin();
                const int b = batch_of[j];
                const int hs = __builtin_popcountll((k ^ xh) & (phys[i].zmask >> c)) & 1;
                PauliDev& d = hd[toff[b] + k * tcnt[b] + fill[b]++];
                d = pauli_dev(phys[i], phys[i].xmask & lowmask, phys[i].zmask & lowmask, 0, hs ? -1.0 : 1.0);
                d.pad = d_full ? (int32_t)(k ^ xh) : slot_of[j];
            }
        }
        if ((e = cudaMemcpy(d_terms, hd.data(), sizeof(PauliDev) * hd.size(), cudaMemcpyHostToDevice)))
            return cuda_fail(s, e, "upload terms");
    }
    if (d_full) {
        // psi decoded once, group by group through the two staging sets
        for (uint64_t k0 = 0, bi = 0; k0 < nch; k0 += gcap, bi++) {
            const int sl = (int)(bi & 1);
            const uint64_t mm = std::min<uint64_t>(gcap, nch - k0);
            if (bi >= 2 && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_h2d[2 + sl], 0)))
                return cuda_fail(s, e, "wait decode");
            GroupIn gin{};
            for (uint64_t j = 0; j < mm; j++) {
                const ChunkRef& cr = s->cur[k0 + j];
                gin.bytes[j] = (uint32_t)cr.bytes;
                if ((e = cudaMemcpyAsync(s->d_in[sl] + j * s->stride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice,
                                         s->s_h2d)))
                    return cuda_fail(s, e, "H2D chunk");
                s->st.bytes_h2d += cr.bytes;
            }
            if ((e = cudaEventRecord(s->ev_h2d[sl], s->s_h2d)) || (e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[sl], 0)) ||
                (e = launch_decode<R>(s->d_in[sl], s->stride, c, s->dtype, (int)mm, gin,
                                      static_cast<uint8_t*>(d_full) + ((k0 << c) * amp_bytes), s->scale, s->d_err,
                                      s->s_comp)) ||
                (e = cudaEventRecord(s->ev_h2d[2 + sl], s->s_comp)))
                return cuda_fail(s, e, "decode psi");
            s->st.kernel_launches++;
        }
    }
    // Every source chunk serves X.size() output chunks. When the whole
    // compressed psi fits beside the staging buffers, it crosses the host
    // link once into a device copy (chunk k at k * cstride) and each output
    // chunk's sources are gathered from there on the device; otherwise each
    // output chunk copies its sources from the host store.
    uint8_t* d_cache = nullptr;
    uint64_t* d_cbytes = nullptr;
    size_t cstride = 0;
    if (!d_full && s->cfg.lambda_cache && X.size() > 1 && nch <= 65536) {
        for (const ChunkRef& cr : s->cur) cstride = std::max<size_t>(cstride, cr.bytes);
        cstride = (cstride + 255) & ~size_t(255);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        cudaGetLastError();
        const bool fits = s->cfg.device_alloc || (double)cstride * nch <= 0.5 * (double)free_b;
        if (fits && (dev_alloc(s, &d_cache, cstride * nch) || dev_alloc(s, &d_cbytes, sizeof(uint64_t) * nch))) {
            cudaGetLastError();
            dev_free(s, d_cache);
            dev_free(s, d_cbytes);
            d_cache = nullptr;
            d_cbytes = nullptr;
        }
        if (d_cache) {
            std::vector<uint64_t> lens(nch);
            for (uint64_t k = 0; k < nch; k++) {
                const ChunkRef& cr = s->cur[k];
                lens[k] = cr.bytes;
                if ((e = cudaMemcpyAsync(d_cache + k * cstride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice, s->s_h2d)))
                    return cuda_fail(s, e, "H2D psi cache");
                s->st.bytes_h2d += cr.bytes;
            }
            if ((e = cudaMemcpyAsync(d_cbytes, lens.data(), sizeof(uint64_t) * nch, cudaMemcpyHostToDevice,
                                     s->s_h2d)) ||
                (e = cudaEventRecord(s->ev_h2d[0], s->s_h2d)) || (e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[0], 0)) ||
                (e = cudaStreamSynchronize(s->s_h2d)))  // lens is a host temporary
                return cuda_fail(s, e, "H2D psi cache");
        }
    }
    struct CacheFree {
        sv_state* s;
        uint8_t*& a;
        uint64_t*& b;
        ~CacheFree()
        {
            if (a || b) {
                cudaStreamSynchronize(s->s_comp);  // the gathers that read them
                dev_free(s, a);
                dev_free(s, b);
            }
        }
    } cache_free{s, d_cache, d_cbytes};
    auto issue = [&](uint64_t k) -> int {
        const int sl = nset == 2 ? (int)(k & 1) : 0;
        const size_t base = (size_t)sl * m;
        uint8_t* in = s->d_in[0] + base * s->stride;
        uint8_t* amps = static_cast<uint8_t*>(s->d_amps) + (base << c) * amp_bytes;
        int launches = 0;
        if (d_full) {
            // the set's output stream is overwritten once its copy to the host is done
            if (k >= (uint64_t)nset && (e = cudaStreamWaitEvent(s->s_comp, s->ev_d2h[sl], 0)))
                return cuda_fail(s, e, "wait d2h");
            if ((e = launch_ham_chunk<R>(d_full, s->d_amps2, c, d_terms + k * nt, (int)nt, 0, s->s_comp)))
                return cuda_fail(s, e, "lambda chunk");
            launches++;
            amps = static_cast<uint8_t*>(d_full) + (k << c) * amp_bytes;  // psi_k
        }
        for (size_t b = 0; b < (d_full ? 0 : nb); b++) {
            GroupIn gin{};
            if (d_cache) {
                // sources from the device copy of psi (compute stream: after the set's previous decode)
                StreamMoves mv;
                for (size_t i = 0; i < batch[b].size(); i++) {
                    const uint64_t src = k ^ X[batch[b][i]];
                    gin.bytes[i] = (uint32_t)s->cur[src].bytes;
                    mv.src[mv.n] = (uint16_t)src;
                    mv.dst[mv.n] = (uint16_t)i;
                    mv.n++;
                }
                if ((e = launch_gather_streams(d_cache, d_cbytes, cstride, in, s->stride, mv, s->s_comp)))
                    return cuda_fail(s, e, "gather sources");
                launches++;
            } else {
                // the set's streams are overwritten once its previous decode is done
                if ((k >= (uint64_t)nset || b > 0) && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_h2d[2 + sl], 0)))
                    return cuda_fail(s, e, "wait decode");
                for (size_t i = 0; i < batch[b].size(); i++) {
                    const ChunkRef& cr = s->cur[k ^ X[batch[b][i]]];
                    gin.bytes[i] = (uint32_t)cr.bytes;
                    if ((e = cudaMemcpyAsync(in + i * s->stride, cr.ptr, cr.bytes, cudaMemcpyHostToDevice, s->s_h2d)))
                        return cuda_fail(s, e, "H2D chunk");
                    s->st.bytes_h2d += cr.bytes;
                }
                if ((e = cudaEventRecord(s->ev_h2d[sl], s->s_h2d)) ||
                    (e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[sl], 0)))
                    return cuda_fail(s, e, "record h2d");
            }
            if ((e = launch_decode<R>(in, s->stride, c, s->dtype, (int)batch[b].size(), gin, amps, s->scale, s->d_err,
                                      s->s_comp)) ||
                (e = cudaEventRecord(s->ev_h2d[2 + sl], s->s_comp)))
                return cuda_fail(s, e, "decode");
            // the set's output stream is overwritten once its copy to the host is done
            if (b == 0 && k >= (uint64_t)nset && (e = cudaStreamWaitEvent(s->s_comp, s->ev_d2h[sl], 0)))
                return cuda_fail(s, e, "wait d2h");
            if ((e = launch_ham_chunk<R>(amps, s->d_amps2, c, d_terms + toff[b] + k * tcnt[b], (int)tcnt[b], b > 0,
                                         s->s_comp)))
                return cuda_fail(s, e, "lambda chunk");
            launches += 2;
        }
        // psi_k: slot 0 of the last batch, or its place in the decoded psi
        if ((e = launch_dot<R>(amps, s->d_amps2, 1ull << c, d_part, nblocks, s->s_comp)) ||
            (e = launch_sum_partials(d_part, 1, nblocks, d_energy, s->s_comp)) ||
            (s->rel && (e = launch_chunk_steps<R>(s->d_amps2, c, 1, s->eb, s->d_mbits, s->d_kc, s->s_comp,
                                                  &launches))) ||
            (e = launch_encode<R>(s->d_amps2, c, s->dtype, s->kl, 1, s->d_out2[sl], s->stride, s->d_sparse,
                                  s->d_blocksq, s->d_co2[sl], s->d_err, s->s_comp, &launches,
                                  s->rel ? s->d_kc : nullptr)) ||
            (e = cudaMemcpyAsync(s->h_co2[sl], s->d_co2[sl], sizeof(ChunkOut), cudaMemcpyDeviceToHost, s->s_comp)) ||
            (e = cudaEventRecord(s->ev_comp[sl], s->s_comp)))
            return cuda_fail(s, e, "lambda chunk");
        s->st.kernel_launches += 2 + launches;
        return SV_OK;
    };
    auto finish = [&](uint64_t k) -> int {
        const int sl = nset == 2 ? (int)(k & 1) : 0;
        int r = wait_event(s, s->ev_comp[sl]);
        if (r) return r;
        const uint64_t bytes = s->h_co2[sl][0].bytes;
        if (bytes > s->stride) return fail(s, SV_ERR_CORRUPT, "encoded chunk larger than its slot");
        uint8_t* dst = store_slot(s, s->lpool, s->lcur[k], bytes);
        if (!dst) return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the lambda store failed");
        if ((e = cudaMemcpyAsync(dst, s->d_out2[sl], bytes, cudaMemcpyDeviceToHost, s->s_d2h)) ||
            (e = cudaEventRecord(s->ev_d2h[sl], s->s_d2h)))
            return cuda_fail(s, e, "D2H lambda chunk");
        s->st.bytes_d2h += bytes;
        return SV_OK;
    };
    int r = SV_OK;
    for (uint64_t k = 0; k < nch && !r; k++) {
        // one set: chunk k's sizes are read before chunk k+1 overwrites them
        if (nset == 1) {
            if (!(r = issue(k))) r = finish(k);
            continue;
        }
        if (!(r = issue(k)) && k >= 1) r = finish(k - 1);
    }
    if (!r && nset == 2 && nch >= 1) r = finish(nch - 1);
    const int rs = sync_all(s);
    return r ? r : rs;
}

// One reverse pass over (psi, lambda): gradient partials and U^dagger on both.
template <typename R>
static int run_pass_adjoint_compressed(sv_state* s, const std::vector<PGate>& inv, const PassPlan& pp,
                                       double* d_gpart, size_t gpart_cap, double* d_acc,
                                       std::vector<int>& slot_params)
{
    const int c = s->c, g = (int)pp.S.size();
    const int L = c + g;
    int t, l;
    tile_shape(L, std::min(s->tq, 12), s->lq, t, l);
    std::vector<int> rids(pp.gates.rbegin(), pp.gates.rend());
    for (int gi : rids) {
        // a partial is evaluated on the tile: the target must be in the pass's group
        const int q = inv[gi].t[0];
        if (inv[gi].param >= 0 && q >= c && std::find(pp.S.begin(), pp.S.end(), q) == pp.S.end())
            return fail(s, SV_ERR_ARG, "parameterised gate on a qubit its pass does not stage");
    }
    const std::vector<HOp> hops = local_ops(inv, rids, c, pp.S, true);
    const std::vector<SubPlan> subs = plan_subpasses(hops, L, t, l, true);
    if (subs.empty() && !hops.empty()) return fail(s, SV_ERR_ARG, "no tile plan for the pass");
    AdjPlan<R> ap;
    int r = jit_adjoint_plan<R>(s, subs, L, t, l, slot_params, ap);
    if (r) return r;
    std::vector<TileDesc> tds;
    std::vector<int> offs, cnts, gslot, nsl;
    std::vector<DevOp<R>> ops;
    if (ap.ok) {
        tds = ap.td;
        gslot = ap.gslot;
        nsl = ap.nsl;
    } else {
        for (const SubPlan& sp : subs) {
            TileDesc td = tile_desc(sp.T, L, t, l);
            tds.push_back(td);
            offs.push_back((int)ops.size());
            gslot.push_back((int)slot_params.size());
            int base = 0;
            dev_ops<R>(sp, td, ops, &base, &slot_params);
            nsl.push_back(base);
            cnts.push_back((int)ops.size() - offs.back());
        }
    }
    const uint64_t ntiles = 1ull << (L - t);
    for (int v : nsl)
        if ((uint64_t)v * ntiles > gpart_cap) return fail(s, SV_ERR_ARG, "gradient partial buffer too small");
    if (!ap.ok && (r = upload_ops<R>(s, ops))) return r;
    const DevOp<R>* d_ops = static_cast<const DevOp<R>*>(s->d_ops);

    std::vector<int> spos, fpos;
    for (int q = c; q < s->n; q++) {
        if (std::find(pp.S.begin(), pp.S.end(), q) != pp.S.end()) spos.push_back(q - c);
        else fpos.push_back(q - c);
    }
    const uint64_t ngroups = 1ull << fpos.size();
    const int gch = 1 << g;
    const int NS = s->nslots;
    std::vector<std::vector<uint64_t>> slot_chunks(NS);

    auto issue = [&](uint64_t gi) -> int {
        const int slot = (int)(gi % NS);
        const uint64_t base = deposit(gi, fpos);
        auto& ch = slot_chunks[slot];
        ch.resize(gch);
        GroupIn gp{}, gl{};
        cudaError_t e;
        if (s->slot_used[slot] && (e = cudaStreamWaitEvent(s->s_h2d, s->ev_comp[slot], 0)))
            return cuda_fail(s, e, "wait comp");
        const int ph2d = prof_begin(s, s->s_h2d);
        for (int j = 0; j < gch; j++) {
            const uint64_t k = base | deposit((uint64_t)j, spos);
            ch[j] = k;
            gp.bytes[j] = (uint32_t)s->cur[k].bytes;
            gl.bytes[j] = (uint32_t)s->lcur[k].bytes;
            if ((e = cudaMemcpyAsync(s->d_in[slot] + (size_t)j * s->stride, s->cur[k].ptr, s->cur[k].bytes,
                                     cudaMemcpyHostToDevice, s->s_h2d)) ||
                (e = cudaMemcpyAsync(s->d_in2[slot] + (size_t)j * s->stride, s->lcur[k].ptr, s->lcur[k].bytes,
                                     cudaMemcpyHostToDevice, s->s_h2d)))
                return cuda_fail(s, e, "H2D chunk");
            s->st.bytes_h2d += s->cur[k].bytes + s->lcur[k].bytes;
        }
        prof_end(s, ph2d, PROF_H2D, 0, s->s_h2d);
        if ((e = cudaEventRecord(s->ev_h2d[slot], s->s_h2d)) || (e = cudaStreamWaitEvent(s->s_comp, s->ev_h2d[slot], 0)))
            return cuda_fail(s, e, "record h2d");
        if (s->slot_used[slot] && (e = cudaStreamWaitEvent(s->s_comp, s->ev_d2h[slot], 0)))
            return cuda_fail(s, e, "wait d2h");
        const uint64_t amp_bytes = (sizeof(R) * 2ull) << L;
        int pi = prof_begin(s);
        if ((e = launch_decode<R>(s->d_in[slot], s->stride, c, s->dtype, gch, gp, s->d_amps, 1.0, s->d_err, s->s_comp)) ||
            (e = launch_decode<R>(s->d_in2[slot], s->stride, c, s->dtype, gch, gl, s->d_amps2, 1.0, s->d_err,
                                  s->s_comp)))
            return cuda_fail(s, e, "decode");
        prof_end(s, pi, PROF_DECODE, 2 * amp_bytes);
        s->st.kernel_launches += 2;
        const uint64_t gbase = base << c;
        for (size_t i = 0; i < tds.size(); i++) {
            pi = prof_begin(s);
            unsigned parts = (unsigned)ntiles;  // gradient partials per slot
            if (ap.ok) {
                e = jit_launch_adjoint<R>(ap.fn[i], s->d_amps, s->d_amps2, tds[i], gbase, d_gpart, ap.par[i], s->s_comp,
                                          &parts);
                s->st.jit_launches++;
                s->st.jit_adjoint_launches++;
            } else {
                e = launch_adjoint<R>(s->d_amps, s->d_amps2, tds[i], d_ops + offs[i], cnts[i], gbase, d_gpart, ntiles,
                                      s->s_comp);
            }
            if (e) return cuda_fail(s, e, "adjoint");
            prof_end(s, pi, PROF_APPLY, 4 * amp_bytes);
            s->st.kernel_launches++;
            if (nsl[i] > 0) {
                if ((e = launch_sum_partials(d_gpart, nsl[i], (int)parts, d_acc + 1 + gslot[i], s->s_comp)))
                    return cuda_fail(s, e, "grad reduce");
                s->st.kernel_launches++;
            }
        }
        int launches = 0;
        pi = prof_begin(s);
        int32_t* kc = s->rel ? s->d_kc : nullptr;
        if ((s->rel && (e = launch_chunk_steps<R>(s->d_amps, c, gch, s->eb, s->d_mbits, s->d_kc, s->s_comp,
                                                  &launches))) ||
            (e = launch_encode<R>(s->d_amps, c, s->dtype, s->k, gch, s->d_out[slot], s->stride, s->d_sparse,
                                  s->d_blocksq, s->d_co[slot], s->d_err, s->s_comp, &launches, kc)) ||
            (s->rel && (e = launch_chunk_steps<R>(s->d_amps2, c, gch, s->eb, s->d_mbits, s->d_kc, s->s_comp,
                                                  &launches))) ||
            (e = launch_encode<R>(s->d_amps2, c, s->dtype, s->kl, gch, s->d_out2[slot], s->stride, s->d_sparse,
                                  s->d_blocksq, s->d_co2[slot], s->d_err, s->s_comp, &launches, kc)))
            return cuda_fail(s, e, "encode");
        prof_end(s, pi, PROF_ENCODE, 2 * amp_bytes);
        if ((e = cudaMemcpyAsync(s->h_co[slot], s->d_co[slot], sizeof(ChunkOut) * gch, cudaMemcpyDeviceToHost,
                                 s->s_comp)) ||
            (e = cudaMemcpyAsync(s->h_co2[slot], s->d_co2[slot], sizeof(ChunkOut) * gch, cudaMemcpyDeviceToHost,
                                 s->s_comp)) ||
            (e = cudaEventRecord(s->ev_comp[slot], s->s_comp)))
            return cuda_fail(s, e, "encode sizes");
        s->st.kernel_launches += launches;
        s->slot_used[slot] = true;
        s->st.groups++;
        s->st.subpasses += tds.size();
        return SV_OK;
    };
    auto finish = [&](uint64_t gi) -> int {
        const int slot = (int)(gi % NS);
        int rr = wait_event(s, s->ev_comp[slot]);
        if (rr) return rr;
        cudaError_t e;
        const int pd2h = prof_begin(s, s->s_d2h);
        for (int j = 0; j < gch; j++) {
            const uint64_t k = slot_chunks[slot][j];
            const ChunkOut cp = s->h_co[slot][j], cl = s->h_co2[slot][j];
            if (cp.bytes > s->stride || cl.bytes > s->stride)
                return fail(s, SV_ERR_CORRUPT, "encoded chunk larger than its slot");
            // both old streams reached the device before the group's compute event
            uint8_t* dp = store_slot(s, s->pool, s->cur[k], cp.bytes);
            uint8_t* dl = store_slot(s, s->lpool, s->lcur[k], cl.bytes);
            if (!dp || !dl) return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the compressed store failed");
            if ((e = cudaMemcpyAsync(dp, s->d_out[slot] + (size_t)j * s->stride, cp.bytes, cudaMemcpyDeviceToHost,
                                     s->s_d2h)) ||
                (e = cudaMemcpyAsync(dl, s->d_out2[slot] + (size_t)j * s->stride, cl.bytes, cudaMemcpyDeviceToHost,
                                     s->s_d2h)))
                return cuda_fail(s, e, "D2H chunk");
            s->st.bytes_d2h += cp.bytes + cl.bytes;
        }
        prof_end(s, pd2h, PROF_D2H, 0, s->s_d2h);
        if ((e = cudaEventRecord(s->ev_d2h[slot], s->s_d2h))) return cuda_fail(s, e, "record d2h");
        return SV_OK;
    };
    for (uint64_t gi = 0; gi <= ngroups; gi++) {
        if (gi < ngroups && (r = issue(gi))) return r;
        if (gi >= 1 && (r = finish(gi - 1))) return r;
    }
    if ((r = sync_all(s))) return r;
    prof_collect(s);
    if ((r = check_device_error(s))) return r;
    s->st.passes++;
    return SV_OK;
}

// psi checkpoints of the compressed adjoint: a copy of every chunk stream of
// the store, taken and put back with host threads (no GPU work is in flight
// on the store at either point: the passes around them have synchronised).
using Checkpoint = std::vector<std::vector<uint8_t>>;

static void parallel_chunks(uint64_t nch, const std::function<void(uint64_t)>& fn)
{
    const uint64_t nth = std::min<uint64_t>(nch, std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    std::atomic<uint64_t> next{0};
    auto worker = [&]() {
        for (uint64_t k; (k = next.fetch_add(1)) < nch;) fn(k);
    };
    std::vector<std::thread> pool;
    for (uint64_t i = 1; i < nth; i++) pool.emplace_back(worker);
    worker();
    for (std::thread& th : pool) th.join();
}

static void checkpoint_take(sv_state* s, Checkpoint& cp)
{
    cp.assign(s->cur.size(), {});
    parallel_chunks(s->cur.size(), [&](uint64_t k) {
        cp[k].assign(s->cur[k].ptr, s->cur[k].ptr + s->cur[k].bytes);
    });
}

static int checkpoint_restore(sv_state* s, const Checkpoint& cp)
{
    // slots first (the pool is not thread-safe), then the copies
    for (uint64_t k = 0; k < cp.size(); k++)
        if (!store_slot(s, s->pool, s->cur[k], cp[k].size()))
            return fail(s, SV_ERR_HOST_OOM, "pinned host allocation for the compressed store failed");
    parallel_chunks(cp.size(), [&](uint64_t k) { std::memcpy(s->cur[k].ptr, cp[k].data(), cp[k].size()); });
    return SV_OK;
}

template <typename R>
int grad_compressed(sv_state* s, const std::vector<PGate>& gates, size_t nparams, const sv_pauli_term* H,
                    size_t nterms, double* energy, double* grad)
{
    int r = ensure_lambda_store<R>(s);
    if (r) return r;
    if ((r = init_state<R>(s))) return r;
    const std::vector<PassPlan> passes = plan_passes(gates, s->n, s->c, s->gmax);
    // the forward sweep (the same plan); with checkpoints pass by pass, keeping
    // psi after every K-th pass (ckpt[i]: psi after (i + 1) K passes)
    const auto tf0 = std::chrono::steady_clock::now();
    const size_t K = (size_t)std::max(0, s->cfg.checkpoint_passes);
    std::vector<Checkpoint> ckpt;
    s->st.checkpoint_bytes = 0;
    s->st.checkpoints = 0;
    if (K == 0 || passes.size() <= K) {
        if ((r = apply_circuit<R>(s, gates, false))) return r;
    } else {
        for (size_t p = 0; p < passes.size(); p++) {
            if ((r = run_pass_compressed<R>(s, gates, passes[p]))) return r;
            if ((p + 1) % K == 0 && p + 1 < passes.size()) {
                ckpt.emplace_back();
                checkpoint_take(s, ckpt.back());
                for (const auto& v : ckpt.back()) s->st.checkpoint_bytes += v.size();
                s->st.checkpoints++;
            }
        }
    }
    std::vector<sv_pauli_term> phys(nterms);
    for (size_t i = 0; i < nterms; i++) {
        phys[i] = H[i];
        phys[i].xmask = mask_to_physical(s->perm, H[i].xmask);
        phys[i].zmask = mask_to_physical(s->perm, H[i].zmask);
    }
    std::vector<PGate> inv(gates.size());
    size_t nparam_gates = 0;
    for (size_t i = 0; i < gates.size(); i++) {
        inv[i] = gates[i];
        const int K = 1 << gates[i].nt;
        for (int a = 0; a < K; a++)
            for (int b = 0; b < K; b++) inv[i].m[a * K + b] = std::conj(gates[i].m[b * K + a]);
        if (gates[i].param >= 0) nparam_gates++;
    }
    const int nblocks = reduce_blocks_for(1ull << s->c);
    const int L = s->c + std::min(s->gmax, s->nh);
    int t, l;
    tile_shape(L, std::min(s->tq, 12), s->lq, t, l);
    const size_t gpart_cap = std::max<size_t>(1, nparam_gates) << (L - t);
    PauliDev* d_terms = nullptr;
    double *d_part = nullptr, *d_acc = nullptr, *d_gpart = nullptr;
    cudaError_t e;
    if ((e = dev_alloc(s, &d_terms, sizeof(PauliDev) * std::max<size_t>(1, nterms) << s->nh)) ||
        (e = dev_alloc(s, &d_part, sizeof(double) * nblocks)) ||
        (e = dev_alloc(s, &d_acc, sizeof(double) * (1 + std::max<size_t>(1, nparam_gates)))) ||
        (e = dev_alloc(s, &d_gpart, sizeof(double) * gpart_cap))) {
        dev_free(s, d_terms); dev_free(s, d_part); dev_free(s, d_acc); dev_free(s, d_gpart);
        return cuda_fail(s, e, "cudaMalloc(grad)");
    }
    std::vector<int> slot_params;
    do {
        cudaMemsetAsync(d_acc, 0, sizeof(double) * (1 + std::max<size_t>(1, nparam_gates)), s->s_comp);
        // lambda = H psi has |lambda_i| <= ||H|| <= sum |c|: its store quantises with the
        // step scaled by the next power of two of sum |c|, keeping q in range
        double csum = 0;
        for (size_t i = 0; i < nterms; i++) csum += std::fabs(H[i].coeff);
        int up = 0;
        while (std::ldexp(1.0, up) < csum && up < 40) up++;
        s->kl = std::min(0, s->k + up);
        const auto tl0 = std::chrono::steady_clock::now();
        s->st.t_grad_forward_s = std::chrono::duration<double>(tl0 - tf0).count();
        if ((r = build_lambda<R>(s, phys, d_terms, d_part, nblocks, d_acc))) break;
        const auto tr0 = std::chrono::steady_clock::now();
        s->st.t_grad_lambda_s = std::chrono::duration<double>(tr0 - tl0).count();
        for (size_t p = passes.size(); p-- > 0;) {
            if ((r = run_pass_adjoint_compressed<R>(s, inv, passes[p], d_gpart, gpart_cap, d_acc, slot_params)))
                break;
            // psi after p passes, as the forward sweep left it, replaces the uncomputed one
            if (K && p > 0 && p % K == 0 && p / K - 1 < ckpt.size() && (r = checkpoint_restore(s, ckpt[p / K - 1])))
                break;
        }
        if (r) break;
        std::vector<double> acc(1 + slot_params.size());
        if ((e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, s->s_comp))) {
            r = cuda_fail(s, e, "D2H grad");
            break;
        }
        if ((r = wait_stream(s, s->s_comp))) break;
        s->st.t_grad_reverse_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - tr0).count();
        *energy = acc[0];
        for (size_t p = 0; p < nparams; p++) grad[p] = 0;
        for (size_t j = 0; j < slot_params.size(); j++) grad[slot_params[j]] += acc[1 + j];
    } while (0);
    dev_free(s, d_terms);
    dev_free(s, d_part);
    dev_free(s, d_acc);
    dev_free(s, d_gpart);
    if (!r) r = check_device_error(s);
    return r;
}

template int grad_compressed<float>(sv_state*, const std::vector<PGate>&, size_t, const sv_pauli_term*, size_t,
                                    double*, double*);
template int grad_compressed<double>(sv_state*, const std::vector<PGate>&, size_t, const sv_pauli_term*, size_t,
                                     double*, double*);
template int apply_circuit<float>(sv_state*, const std::vector<PGate>&, bool);
template int apply_circuit<double>(sv_state*, const std::vector<PGate>&, bool);
template int jit_sources<float>(sv_state*, const std::vector<PGate>&, std::vector<std::string>&, bool);
template int jit_sources<double>(sv_state*, const std::vector<PGate>&, std::vector<std::string>&, bool);
template int init_state<float>(sv_state*);
template int init_state<double>(sv_state*);
template int amplitudes<float>(sv_state*, const uint64_t*, size_t, double*);
template int inner<float, float>(sv_state*, const sv_state*, double*);
template int inner<float, double>(sv_state*, const sv_state*, double*);
template int inner<double, float>(sv_state*, const sv_state*, double*);
template int inner<double, double>(sv_state*, const sv_state*, double*);
template int amplitudes<double>(sv_state*, const uint64_t*, size_t, double*);
template int expect<float>(sv_state*, const sv_pauli_term*, size_t, double*);
template int expect<double>(sv_state*, const sv_pauli_term*, size_t, double*);
template int grad_uncompressed<float>(sv_state*, const std::vector<PGate>&, size_t, const sv_pauli_term*, size_t,
                                      double*, double*);
template int grad_uncompressed<double>(sv_state*, const std::vector<PGate>&, size_t, const sv_pauli_term*, size_t,
                                       double*, double*);

}  // namespace sv
