// api.cpp -- the C ABI of include/sv.h: argument validation, handle life
// cycle, SWAP absorption into the logical->physical qubit map, and dispatch
// to the complex64 / complex128 engines.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "engine.h"

using namespace sv;

namespace {

thread_local std::string g_create_error;

// Calls that apply gates use the module's constant-memory op tables: they
// run one at a time per process (each call is synchronous).
std::mutex g_apply_mu;

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int step_exponent(double eb)
{
    int e = 0;
    std::frexp(2.0 * eb, &e);  // 2 eb = m 2^e, m in [0.5, 1)
    return e - 1;
}

// Validate one gate against n qubits; fills g (targets/controls already physical).
int validate_gate(const sv_gate& in, int n, bool allow_param, std::string& why)
{
    if (in.kind > SV_GATE_CUSTOM) { why = "unknown gate kind"; return SV_ERR_ARG; }
    if (in.ntargets < 1 || in.ntargets > 2 || in.ncontrols > 2) { why = "bad target/control count"; return SV_ERR_ARG; }
    const int k = (int)in.kind;
    if (k == SV_GATE_SWAP && in.ntargets != 2) { why = "SWAP needs 2 targets"; return SV_ERR_ARG; }
    if (k != SV_GATE_SWAP && k != SV_GATE_CUSTOM && in.ntargets != 1) { why = "gate takes one target"; return SV_ERR_ARG; }
    if ((k == SV_GATE_CNOT || k == SV_GATE_CZ || k == SV_GATE_CP) && in.ncontrols < 1) {
        why = "controlled gate without control";
        return SV_ERR_ARG;
    }
    if (k == SV_GATE_SWAP && in.ncontrols) { why = "controlled SWAP not supported"; return SV_ERR_ARG; }
    uint64_t seen = 0;
    for (uint32_t i = 0; i < in.ntargets + in.ncontrols; i++) {
        const uint32_t q = i < in.ntargets ? in.targets[i] : in.controls[i - in.ntargets];
        if ((int)q >= n) { why = "qubit out of range"; return SV_ERR_ARG; }
        if (seen & (1ull << q)) { why = "repeated qubit in a gate"; return SV_ERR_ARG; }
        seen |= 1ull << q;
    }
    if (!std::isfinite(in.theta)) { why = "angle not finite"; return SV_ERR_ARG; }
    if (k == SV_GATE_CUSTOM) {
        const int K = 1 << in.ntargets;
        for (int i = 0; i < 2 * K * K; i++)
            if (!std::isfinite(in.mat[i])) { why = "custom matrix not finite"; return SV_ERR_ARG; }
    }
    if (allow_param && in.param_index >= 0) {
        if ((k != SV_GATE_RX && k != SV_GATE_RY && k != SV_GATE_RZ) || in.ncontrols) {
            why = "parameterised gates must be uncontrolled RX, RY or RZ";
            return SV_ERR_ARG;
        }
    }
    return SV_OK;
}

// Lower the gate list onto physical qubits: SWAPs update perm, other gates
// are mapped through it. theta (if non-null) overrides parameterised angles.
int lower(sv_state* s, const sv_gate* gates, size_t ngates, const double* theta, size_t nparams, bool grad,
          std::vector<PGate>& out)
{
    std::string why;
    for (size_t i = 0; i < ngates; i++) {
        if (validate_gate(gates[i], s->n, grad, why)) return fail(s, SV_ERR_ARG, "gate " + std::to_string(i) + ": " + why);
        if (grad && gates[i].param_index >= 0 && (size_t)gates[i].param_index >= nparams)
            return fail(s, SV_ERR_ARG, "gate " + std::to_string(i) + ": parameter index out of range");
    }
    out.clear();
    out.reserve(ngates);
    for (size_t i = 0; i < ngates; i++) {
        const sv_gate& in = gates[i];
        if (in.kind == SV_GATE_SWAP) {
            std::swap(s->perm[in.targets[0]], s->perm[in.targets[1]]);
            continue;
        }
        PGate g;
        g.kind = (int)in.kind;
        g.nt = (int)in.ntargets;
        g.nc = (int)in.ncontrols;
        for (int j = 0; j < g.nt; j++) g.t[j] = s->perm[in.targets[j]];
        for (int j = 0; j < g.nc; j++) g.c[j] = s->perm[in.controls[j]];
        g.theta = in.theta;
        g.param = grad ? in.param_index : -1;
        if (grad && in.param_index >= 0 && theta) g.theta = theta[in.param_index];
        gate_matrix(g.kind, g.theta, in.mat, g.nt, g.m);
        g.diag = kind_is_diag(g.kind);
        if (g.kind == SV_GATE_CUSTOM) {
            const int K = 1 << g.nt;
            bool d = true;
            for (int a = 0; a < K; a++)
                for (int b = 0; b < K; b++)
                    if (a != b && g.m[a * K + b] != cd(0, 0)) d = false;
            g.diag = d;
        }
        out.push_back(g);
    }
    return SV_OK;
}

// A handle call's GPU work starts after the work the caller queued on its
// stream before the call, and the caller's stream waits for the call's work.
struct CallOrder {
    sv_state* s;
    explicit CallOrder(sv_state* st) : s(st)
    {
        if (!s || !s->cfg.stream || !s->ev_user) return;
        cudaStream_t u = static_cast<cudaStream_t>(s->cfg.stream);
        if (cudaEventRecord(s->ev_user, u) == cudaSuccess) {
            cudaStreamWaitEvent(s->s_comp, s->ev_user, 0);
            cudaStreamWaitEvent(s->s_h2d, s->ev_user, 0);
            cudaStreamWaitEvent(s->s_d2h, s->ev_user, 0);
        }
        cudaGetLastError();
    }
    ~CallOrder()
    {
        if (!s || !s->cfg.stream || !s->ev_done) return;
        cudaStream_t u = static_cast<cudaStream_t>(s->cfg.stream);
        // every stream's work joins the compute stream, then the caller's waits on it
        for (cudaStream_t o : {s->s_h2d, s->s_d2h})
            if (cudaEventRecord(s->ev_user, o) == cudaSuccess) cudaStreamWaitEvent(s->s_comp, s->ev_user, 0);
        if (cudaEventRecord(s->ev_done, s->s_comp) == cudaSuccess) cudaStreamWaitEvent(u, s->ev_done, 0);
        cudaGetLastError();
    }
};

void release(sv_state* s)
{
    if (!s) return;
    if (s->s_comp) cudaStreamSynchronize(s->s_comp);
    if (s->s_h2d) cudaStreamSynchronize(s->s_h2d);
    if (s->s_d2h) cudaStreamSynchronize(s->s_d2h);
    if (s->ev_user) cudaEventDestroy(s->ev_user);
    if (s->ev_done) cudaEventDestroy(s->ev_done);
    for (int i = 0; i < 4; i++) {
        dev_free(s, s->d_in[i]);
        dev_free(s, s->d_out[i]);
        dev_free(s, s->d_co[i]);
        if (s->h_co[i]) cudaFreeHost(s->h_co[i]);
        dev_free(s, s->d_in2[i]);
        dev_free(s, s->d_out2[i]);
        dev_free(s, s->d_co2[i]);
        if (s->h_co2[i]) cudaFreeHost(s->h_co2[i]);
        if (s->ev_h2d[i]) cudaEventDestroy(s->ev_h2d[i]);
        if (s->ev_comp[i]) cudaEventDestroy(s->ev_comp[i]);
        if (s->ev_d2h[i]) cudaEventDestroy(s->ev_d2h[i]);
    }
    dev_free(s, s->d_carry);
    dev_free(s, s->d_carry_bytes);
    dev_free(s, s->d_kc);
    dev_free(s, s->d_mbits);
    if (s->ev_prev_d2h) cudaEventDestroy(s->ev_prev_d2h);
    dev_free(s, s->d_amps);
    dev_free(s, s->d_sparse);
    dev_free(s, s->d_blocksq);
    dev_free(s, s->d_err);
    dev_free(s, s->d_state);
    dev_free(s, s->d_lam);
    dev_free(s, s->d_ops);
    for (cudaEvent_t ev : s->prof_ev) cudaEventDestroy(ev);
    dev_free(s, s->d_amps2);
    pool_free(s->pool);
    pool_free(s->lpool);
    if (s->s_comp) cudaStreamDestroy(s->s_comp);
    if (s->s_h2d) cudaStreamDestroy(s->s_h2d);
    if (s->s_d2h) cudaStreamDestroy(s->s_d2h);
    delete s;
}

// Device bytes of the streaming buffers for groups of 2^g chunks (create_impl).
static size_t group_footprint(int c, int g, int dtype, int nslots)
{
    const CodecLayout L = codec_layout(c);
    const size_t stride = (L.max_bytes + 255) & ~size_t(255);
    const size_t amp = dtype == SV_C128 ? 16 : 8;
    const size_t per_chunk = (amp << c) + (size_t)L.nb * 1024 + 8ull * L.bpc +
                             (size_t)nslots * (2 * stride + sizeof(ChunkOut)) + stride;  // + the carry buffer
    return per_chunk << g;
}

// Automatic g_max: the largest group (at most 2^8 chunks) that keeps at least
// four groups per pass for the copy / compute pipeline when the state has
// enough chunks, and whose buffers take at most 40% of the free device memory
// (an adjoint gradient allocates a second set of the same size).
static int auto_group_qubits(int n, int c, const sv_config& cfg)
{
    const int nh = n - c;
    if (cfg.mode != SV_COMPRESSED || nh <= 2) return 2;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    int g = std::max(2, std::min(8, nh >= 4 ? nh - 2 : nh));
    while (g > 2 && group_footprint(c, g, cfg.dtype, cfg.pipeline_slots) > (size_t)(0.4 * (double)free_b)) g--;
    return g;
}

template <typename R>
int create_impl(sv_state* s)
{
    cudaError_t e;
    if ((e = dev_alloc(s, &s->d_err, sizeof(int)))) return cuda_fail(s, e, "cudaMalloc(err)");
    if ((e = cudaMemset(s->d_err, 0, sizeof(int)))) return cuda_fail(s, e, "cudaMemset(err)");
    const size_t amp_bytes = 2 * sizeof(R);
    if (s->mode == SV_UNCOMPRESSED) {
        if ((e = dev_alloc(s, &s->d_state, amp_bytes << s->n)))
            return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the state failed");
        s->st.raw_bytes = amp_bytes << s->n;
        return init_state<R>(s);
    }
    const int gsz = std::min(s->gmax, s->nh);
    const uint64_t gch = 1ull << gsz;
    const CodecLayout L = codec_layout(s->c);
    s->stride = (L.max_bytes + 255) & ~size_t(255);
    if ((e = dev_alloc(s, &s->d_amps, (amp_bytes << s->c) * gch)) ||
        (e = dev_alloc(s, &s->d_sparse, (size_t)L.nb * 1024 * gch)) ||
        (e = dev_alloc(s, &s->d_blocksq, sizeof(unsigned long long) * L.bpc * gch))) {
        cudaGetLastError();
        return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the chunk-group buffers failed");
    }
    for (int i = 0; i < s->nslots; i++) {
        if ((e = dev_alloc(s, &s->d_in[i], s->stride * gch)) || (e = dev_alloc(s, &s->d_out[i], s->stride * gch)) ||
            (e = dev_alloc(s, &s->d_co[i], sizeof(ChunkOut) * gch))) {
            cudaGetLastError();
            return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the staging slots failed");
        }
        if ((e = cudaHostAlloc(&s->h_co[i], sizeof(ChunkOut) * gch, cudaHostAllocDefault)))
            return fail(s, SV_ERR_HOST_OOM, "pinned allocation failed");
    }
    // all four of each (the lambda construction of the adjoint uses events
    // 2 and 3 whatever the slot count)
    for (int i = 0; i < 4; i++)
        if ((e = cudaEventCreateWithFlags(&s->ev_h2d[i], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&s->ev_comp[i], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&s->ev_d2h[i], cudaEventDisableTiming)))
            return cuda_fail(s, e, "cudaEventCreate");
    if ((e = dev_alloc(s, &s->d_kc, sizeof(int32_t) * gch)) || (e = dev_alloc(s, &s->d_mbits, sizeof(uint64_t) * gch))) {
        cudaGetLastError();
        return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the chunk step table failed");
    }
    if ((e = dev_alloc(s, &s->d_carry, s->stride * gch)) || (e = dev_alloc(s, &s->d_carry_bytes, sizeof(uint64_t) * gch))) {
        cudaGetLastError();
        return fail(s, SV_ERR_DEVICE_OOM, "device allocation of the carry buffer failed");
    }
    if ((e = cudaEventCreateWithFlags(&s->ev_prev_d2h, cudaEventDisableTiming))) return cuda_fail(s, e, "cudaEventCreate");
    const uint64_t nchunks = 1ull << s->nh;
    s->carry_at.assign(nchunks, -1);
    s->cur.assign(nchunks, ChunkRef{});
    // pinned segments: an eighth of the raw state, at least four slot strides, at most 4 GiB
    s->pool.seg_bytes = std::min<size_t>((size_t)4 << 30, std::max<size_t>(4 * s->stride, (amp_bytes << s->n) / 8));
    s->st.raw_bytes = amp_bytes << s->n;
    s->st.quant_step = std::ldexp(1.0, s->k);
    return init_state<R>(s);
}

}  // namespace

extern "C" {

void sv_config_default(sv_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->dtype = SV_C64;
    cfg->mode = SV_COMPRESSED;
    cfg->init_index = 0;
    cfg->max_group_qubits = 0;
    cfg->tile_qubits = 0;
    cfg->pipeline_slots = 3;
    cfg->renormalize = 0;
    cfg->device = 0;
    cfg->host_budget_bytes = 0;
    cfg->fuse_codec = 1;
    cfg->jit = 1;
    cfg->relative_bound = 0;
    cfg->remap_qubits = 0;
    cfg->timeout_s = 600.0;
    cfg->checkpoint_passes = 0;
    cfg->lambda_cache = 1;
    cfg->device_alloc = nullptr;
    cfg->device_free = nullptr;
    cfg->alloc_ctx = nullptr;
    cfg->stream = nullptr;
}

int sv_create(int n, int chunk_qubits, double abs_error_bound, const sv_config* cfg_in, sv_state** out)
{
    if (!out) return SV_ERR_ARG;
    *out = nullptr;
    g_create_error.clear();
    sv_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else sv_config_default(&cfg);
    auto reject = [&](int code, const char* msg) {
        g_create_error = msg;
        return code;
    };
    if (n < 1 || n > 40) return reject(SV_ERR_ARG, "n must be in 1..40");
    if (cfg.dtype != SV_C64 && cfg.dtype != SV_C128) return reject(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
    if (cfg.mode != SV_COMPRESSED && cfg.mode != SV_UNCOMPRESSED) return reject(SV_ERR_ARG, "bad mode");
    if (cfg.init_index >> n) return reject(SV_ERR_ARG, "init_index out of range");
    if (cfg.max_group_qubits != 0 && (cfg.max_group_qubits < 2 || cfg.max_group_qubits > 8))
        return reject(SV_ERR_ARG, "max_group_qubits must be 0 (automatic) or 2..8");
    if (cfg.pipeline_slots < 2 || cfg.pipeline_slots > 4) return reject(SV_ERR_ARG, "pipeline_slots must be 2..4");
    if (cfg.tile_qubits && (cfg.tile_qubits < 2 || cfg.tile_qubits > kMaxTileQubits))
        return reject(SV_ERR_ARG, "tile_qubits must be 2..13");
    if (cfg.remap_qubits != 0 && cfg.remap_qubits != 1) return reject(SV_ERR_ARG, "remap_qubits must be 0 or 1");
    if (!(cfg.timeout_s > 0)) cfg.timeout_s = 600.0;
    if (cfg.checkpoint_passes < 0) return reject(SV_ERR_ARG, "checkpoint_passes must be >= 0");
    if (cfg.lambda_cache < 0 || cfg.lambda_cache > 2) return reject(SV_ERR_ARG, "lambda_cache must be 0, 1 or 2");
    if (!cfg.device_alloc != !cfg.device_free)
        return reject(SV_ERR_ARG, "device_alloc and device_free must be set together");
    int k = 0;
    if (cfg.mode == SV_COMPRESSED) {
        if (chunk_qubits < 8 || chunk_qubits > n || chunk_qubits > 30)
            return reject(SV_ERR_ARG, "chunk_qubits must be in 8..min(n, 30)");
        if (!(abs_error_bound > 0) || !std::isfinite(abs_error_bound) || abs_error_bound > 1.0)
            return reject(SV_ERR_ARG, "abs_error_bound must be in (0, 1]");
        k = step_exponent(abs_error_bound);
        const int kmin = cfg.dtype == SV_C64 ? -23 : -29;  // |q| of an amplitude of magnitude 1 must fit
        if (k < kmin) return reject(SV_ERR_RANGE, "abs_error_bound too small for the quantiser's integer range");
        // relative bound: |q| < 1/eb must fit the quantiser
        if (cfg.relative_bound && abs_error_bound < std::ldexp(1.0, kmin))
            return reject(SV_ERR_RANGE, "relative bound: eb below 2^-23 (complex64) / 2^-29 (complex128)");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return reject(SV_ERR_CUDA, "no CUDA device");
    }
    if (cfg.device < 0 || cfg.device >= ndev) return reject(SV_ERR_ARG, "device ordinal out of range");
    if (cudaSetDevice(cfg.device) != cudaSuccess) return reject(SV_ERR_CUDA, "cudaSetDevice failed");

    sv_state* s = new (std::nothrow) sv_state();
    if (!s) return reject(SV_ERR_HOST_OOM, "out of host memory");
    s->n = n;
    s->cfg = cfg;
    s->dtype = cfg.dtype;
    s->mode = cfg.mode;
    s->c = cfg.mode == SV_COMPRESSED ? chunk_qubits : n;
    s->nh = n - s->c;
    s->eb = abs_error_bound;
    s->k = k;
    s->rel = cfg.mode == SV_COMPRESSED && cfg.relative_bound != 0;
    s->gmax = cfg.max_group_qubits ? cfg.max_group_qubits : auto_group_qubits(n, chunk_qubits, cfg);
    s->nslots = cfg.pipeline_slots;
    s->tq = cfg.tile_qubits ? cfg.tile_qubits : kPhaseTileQubits;
    s->lq = kTileLowQubits;
    s->perm.resize(n);
    for (int q = 0; q < n; q++) s->perm[q] = q;
    s->st.chunk_qubits = s->c;
    s->st.group_qubits = std::min(s->gmax, s->nh);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking)) ||
        (e = cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking)) ||
        (e = cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking))) {
        g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
        release(s);
        return SV_ERR_CUDA;
    }
    if (cfg.stream && ((e = cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming)) ||
                       (e = cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming)))) {
        g_create_error = std::string("cudaEventCreate: ") + cudaGetErrorString(e);
        release(s);
        return SV_ERR_CUDA;
    }
    int r;
    {
        CallOrder order(s);
        r = s->dtype == SV_C64 ? create_impl<float>(s) : create_impl<double>(s);
    }
    if (r) {
        g_create_error = s->err;
        release(s);
        return r;
    }
    *out = s;
    return SV_OK;
}

int sv_apply_circuit(sv_state* s, const sv_gate* gates, size_t ngates)
{
    if (!s || (ngates && !gates)) return SV_ERR_ARG;
    s->err.clear();
    const double t0 = now_s();
    const std::vector<int> saved = s->perm;
    std::vector<PGate> pg;
    int r = lower(s, gates, ngates, nullptr, 0, false, pg);
    if (r) {
        s->perm = saved;
        return r;
    }
    cudaSetDevice(s->cfg.device);
    {
        CallOrder order(s);
        std::lock_guard<std::mutex> lock(g_apply_mu);
        const bool remap = s->cfg.remap_qubits != 0;
        r = s->dtype == SV_C64 ? apply_circuit<float>(s, pg, remap) : apply_circuit<double>(s, pg, remap);
    }
    if (!r) {
        s->st.amp_gate_updates += (uint64_t)ngates << s->n;
        s->st.gates_applied += ngates;
    }
    s->st.last_call_seconds = now_s() - t0;
    return r;
}

int sv_expect(sv_state* s, const sv_pauli_term* terms, size_t nterms, double* out_re)
{
    if (!s || !out_re || (nterms && !terms)) return SV_ERR_ARG;
    s->err.clear();
    for (size_t i = 0; i < nterms; i++)
        if (!std::isfinite(terms[i].coeff)) return fail(s, SV_ERR_ARG, "coefficient not finite");
    cudaSetDevice(s->cfg.device);
    CallOrder order(s);
    return s->dtype == SV_C64 ? expect<float>(s, terms, nterms, out_re) : expect<double>(s, terms, nterms, out_re);
}

int sv_amplitudes(sv_state* s, const uint64_t* idx, size_t m, double* out)
{
    if (!s || (m && (!idx || !out))) return SV_ERR_ARG;
    s->err.clear();
    cudaSetDevice(s->cfg.device);
    CallOrder order(s);
    return s->dtype == SV_C64 ? amplitudes<float>(s, idx, m, out) : amplitudes<double>(s, idx, m, out);
}

int sv_inner(sv_state* a, const sv_state* b, double* out_re, double* out_im)
{
    if (!a || !b || !out_re || !out_im) return SV_ERR_ARG;
    a->err.clear();
    if (b->mode != SV_UNCOMPRESSED) return fail(a, SV_ERR_ARG, "sv_inner: the second state must be uncompressed");
    if (a->n != b->n) return fail(a, SV_ERR_ARG, "sv_inner: the states differ in qubit count");
    if (a->cfg.device != b->cfg.device) return fail(a, SV_ERR_ARG, "sv_inner: the states are on different devices");
    cudaSetDevice(a->cfg.device);
    CallOrder order(a);
    double out[2] = {0, 0};
    int r;
    if (a->dtype == SV_C64)
        r = b->dtype == SV_C64 ? inner<float, float>(a, b, out) : inner<float, double>(a, b, out);
    else
        r = b->dtype == SV_C64 ? inner<double, float>(a, b, out) : inner<double, double>(a, b, out);
    if (r) return r;
    *out_re = out[0];
    *out_im = out[1];
    return SV_OK;
}

int sv_device_state(sv_state* s, void** d_amps, int32_t* positions)
{
    if (!s || !d_amps) return SV_ERR_ARG;
    if (s->mode != SV_UNCOMPRESSED) return fail(s, SV_ERR_ARG, "sv_device_state: the state is compressed");
    *d_amps = s->d_state;
    if (positions)
        for (int q = 0; q < s->n; q++) positions[q] = s->perm[q];
    return SV_OK;
}

int sv_amplitudes_range(sv_state* s, uint64_t first, size_t count, double* out)
{
    if (!s || (count && !out)) return SV_ERR_ARG;
    if (count && (first >> s->n || ((first + count - 1) >> s->n) || first + count < first))
        return fail(s, SV_ERR_ARG, "amplitude range out of bounds");
    const size_t batch = (size_t)1 << 22;
    std::vector<uint64_t> idx;
    for (size_t b0 = 0; b0 < count; b0 += batch) {
        const size_t nb = std::min(batch, count - b0);
        idx.resize(nb);
        for (size_t i = 0; i < nb; i++) idx[i] = first + b0 + i;
        const int r = sv_amplitudes(s, idx.data(), nb, out + 2 * b0);
        if (r) return r;
    }
    return SV_OK;
}

int sv_grad(sv_state* s, const sv_gate* gates, size_t ngates, const double* theta, size_t nparams,
            const sv_pauli_term* H, size_t nterms, double* energy, double* grad)
{
    if (!s || (ngates && !gates) || (nparams && !theta) || (nterms && !H) || !energy) return SV_ERR_ARG;
    s->err.clear();
    for (size_t p = 0; p < nparams; p++)
        if (!std::isfinite(theta[p])) return fail(s, SV_ERR_ARG, "theta not finite");
    const double t0 = now_s();
    for (int q = 0; q < s->n; q++) s->perm[q] = q;
    std::vector<PGate> pg;
    int r = lower(s, gates, ngates, theta, nparams, true, pg);
    if (r) return r;
    cudaSetDevice(s->cfg.device);
    CallOrder order(s);
    std::lock_guard<std::mutex> lock(g_apply_mu);
    if (!grad) {
        // energy only: the forward sweep from |init_index> and the expectation
        r = s->dtype == SV_C64 ? init_state<float>(s) : init_state<double>(s);
        if (!r) r = s->dtype == SV_C64 ? apply_circuit<float>(s, pg, false) : apply_circuit<double>(s, pg, false);
        if (!r) r = s->dtype == SV_C64 ? expect<float>(s, H, nterms, energy) : expect<double>(s, H, nterms, energy);
    } else if (s->mode == SV_UNCOMPRESSED)
        r = s->dtype == SV_C64 ? grad_uncompressed<float>(s, pg, nparams, H, nterms, energy, grad)
                               : grad_uncompressed<double>(s, pg, nparams, H, nterms, energy, grad);
    else
        r = s->dtype == SV_C64 ? grad_compressed<float>(s, pg, nparams, H, nterms, energy, grad)
                               : grad_compressed<double>(s, pg, nparams, H, nterms, energy, grad);
    s->st.last_call_seconds = now_s() - t0;
    return r;
}

static int plan_impl(int n, int c, int gmax, int tile_qubits, const sv_gate* gates, size_t ngates, int32_t* order,
                     int32_t* pass_of, uint64_t* staged, size_t* out_executed, size_t* out_passes,
                     size_t* out_subpasses, bool remap, size_t* out_swaps, int32_t* swaps, int32_t* qubits,
                     int32_t* positions)
{
    if (n < 1 || n > 40 || c < 1 || c > n || gmax < 2 || gmax > 8 || (ngates && !gates) || !order || !pass_of ||
        !staged || !out_executed || !out_passes || !out_subpasses || (remap && !out_swaps))
        return SV_ERR_ARG;
    if (tile_qubits && (tile_qubits < 2 || tile_qubits > kMaxTileQubits)) return SV_ERR_ARG;
    sv_state tmp;
    tmp.n = n;
    tmp.perm.resize(n);
    for (int q = 0; q < n; q++) tmp.perm[q] = q;
    std::vector<PGate> input;
    int r = lower(&tmp, gates, ngates, nullptr, 0, false, input);
    if (r) {
        g_create_error = tmp.err;
        return r;
    }
    // index of each lowered gate in the caller's list
    std::vector<int32_t> orig;
    for (size_t i = 0; i < ngates; i++)
        if (gates[i].kind != SV_GATE_SWAP) orig.push_back((int32_t)i);
    std::vector<PGate> pg;
    std::vector<int> where, src;
    const std::vector<PassPlan> passes = plan_circuit(input, n, c, gmax, remap, pg, where, &src);
    size_t k = 0, subs = 0, ns = 0;
    const int tq = tile_qubits ? tile_qubits : 12;
    for (size_t p = 0; p < passes.size(); p++) {
        uint64_t m = 0;
        for (int q : passes[p].S) m |= 1ull << q;
        staged[p] = m;
        for (int gi : passes[p].gates) {
            if (src[gi] < 0) {  // an added SWAP
                if (swaps) {
                    swaps[3 * ns] = (int32_t)p;
                    swaps[3 * ns + 1] = pg[gi].t[0];
                    swaps[3 * ns + 2] = pg[gi].t[1];
                }
                ns++;
                continue;
            }
            order[k] = orig[src[gi]];
            if (qubits) {
                const PGate& G = pg[gi];
                for (int j = 0; j < 2; j++) qubits[4 * k + j] = j < G.nt ? G.t[j] : -1;
                for (int j = 0; j < 2; j++) qubits[4 * k + 2 + j] = j < G.nc ? G.c[j] : -1;
            }
            pass_of[k] = (int32_t)p;
            k++;
        }
        const int L = c + (int)passes[p].S.size();
        int t, l;
        tile_shape(L, tq, kTileLowQubits, t, l);
        const std::vector<HOp> hops = local_ops(pg, passes[p].gates, c, passes[p].S, false);
        const std::vector<SubPlan> sp = plan_subpasses(hops, L, t, l, true);
        if (sp.empty() && !hops.empty()) return SV_ERR_ARG;
        subs += sp.size();
    }
    *out_executed = k;
    *out_passes = passes.size();
    *out_subpasses = subs;
    if (out_swaps) *out_swaps = pg.size() - input.size();
    if (positions)
        for (int q = 0; q < n; q++) positions[q] = where[tmp.perm[q]];
    return SV_OK;
}

int sv_plan(int n, int c, int gmax, int tile_qubits, const sv_gate* gates, size_t ngates, int32_t* order,
            int32_t* pass_of, uint64_t* staged, size_t* out_executed, size_t* out_passes, size_t* out_subpasses)
{
    return plan_impl(n, c, gmax, tile_qubits, gates, ngates, order, pass_of, staged, out_executed, out_passes,
                     out_subpasses, false, nullptr, nullptr, nullptr, nullptr);
}

int sv_plan_remap(int n, int c, int gmax, int tile_qubits, const sv_gate* gates, size_t ngates, int32_t* order,
                  int32_t* pass_of, uint64_t* staged, size_t* out_executed, size_t* out_passes,
                  size_t* out_subpasses, size_t* out_swaps, int32_t* swaps, int32_t* qubits, int32_t* positions)
{
    return plan_impl(n, c, gmax, tile_qubits, gates, ngates, order, pass_of, staged, out_executed, out_passes,
                     out_subpasses, true, out_swaps, swaps, qubits, positions);
}

int sv_jit_sources(int n, int c, const sv_config* cfg_in, const sv_gate* gates, size_t ngates, int adjoint, char* buf,
                   size_t cap, size_t* needed, size_t* nkernels)
{
    sv_config cfg;
    sv_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (n < 1 || n > 40 || (ngates && !gates) || !needed || !nkernels) return SV_ERR_ARG;
    if (cfg.mode == SV_COMPRESSED && (c < 8 || c > n)) return SV_ERR_ARG;
    if (cfg.tile_qubits && (cfg.tile_qubits < 2 || cfg.tile_qubits > kMaxTileQubits)) return SV_ERR_ARG;
    sv_state tmp;
    tmp.n = n;
    tmp.c = cfg.mode == SV_COMPRESSED ? c : n;
    tmp.mode = cfg.mode;
    tmp.dtype = cfg.dtype;
    tmp.cfg = cfg;
    tmp.gmax = cfg.max_group_qubits ? cfg.max_group_qubits : 4;
    tmp.tq = cfg.tile_qubits ? cfg.tile_qubits : kPhaseTileQubits;
    tmp.lq = kTileLowQubits;
    tmp.perm.resize(n);
    for (int q = 0; q < n; q++) tmp.perm[q] = q;
    std::vector<PGate> pg;
    size_t nparams = 0;
    for (size_t i = 0; adjoint && i < ngates; i++)
        if (gates[i].param_index >= 0) nparams = std::max(nparams, (size_t)gates[i].param_index + 1);
    int r = lower(&tmp, gates, ngates, nullptr, nparams, adjoint != 0, pg);
    std::vector<std::string> src;
    if (!r)
        r = cfg.dtype == SV_C128 ? jit_sources<double>(&tmp, pg, src, adjoint != 0)
                                 : jit_sources<float>(&tmp, pg, src, adjoint != 0);
    if (r) {
        g_create_error = tmp.err;
        return r;
    }
    size_t total = 0;
    for (const std::string& x : src) total += x.size() + 1;
    *needed = total;
    *nkernels = src.size();
    if (!buf) return SV_OK;
    if (cap < total) return SV_ERR_ARG;
    for (const std::string& x : src) {
        std::memcpy(buf, x.c_str(), x.size() + 1);
        buf += x.size() + 1;
    }
    return SV_OK;
}

int sv_chunk_stream(const sv_state* s, uint64_t k, void* h_buf, size_t cap, size_t* h_nbytes)
{
    if (!s || !h_nbytes || s->mode != SV_COMPRESSED || k >= s->cur.size()) return SV_ERR_ARG;
    const ChunkRef& cr = s->cur[k];
    *h_nbytes = cr.bytes;
    if (!h_buf || cap < cr.bytes) return SV_ERR_ARG;
    std::memcpy(h_buf, cr.ptr, cr.bytes);
    return SV_OK;
}

int sv_set_profile(sv_state* s, int on)
{
    if (!s) return SV_ERR_ARG;
    s->cfg.profile = on ? 1 : 0;
    return SV_OK;
}

int sv_stats(const sv_state* s, sv_stats_t* out)
{
    if (!s || !out) return SV_ERR_ARG;
    *out = s->st;
    out->host_pinned_bytes = s->pinned_bytes;
    return SV_OK;
}

const char* sv_last_error(const sv_state* s)
{
    if (!s) return g_create_error.c_str();
    return s->err.c_str();
}

void sv_destroy(sv_state* s) { release(s); }

// ------------------------------------------------------------ codec calls
size_t sv_codec_max_bytes(int chunk_qubits)
{
    if (chunk_qubits < 8 || chunk_qubits > 30) return 0;
    return codec_layout(chunk_qubits).max_bytes;
}

static int codec_encode_impl(int dtype, int c, double eb, const void* d_amps, void* d_stream, size_t cap,
                             size_t* h_nbytes, bool relative)
{
    if ((dtype != SV_C64 && dtype != SV_C128) || c < 8 || c > 30 || !d_amps || !d_stream || !h_nbytes)
        return SV_ERR_ARG;
    if (!(eb > 0) || !std::isfinite(eb) || eb > 1.0) return SV_ERR_ARG;
    const int k = step_exponent(eb);
    if (k < -60) return SV_ERR_RANGE;
    // relative bound: |q| < 1/eb must fit the quantiser (2^24 - 1 / 2^30 - 1)
    if (relative && eb < std::ldexp(1.0, dtype == SV_C64 ? -23 : -29)) return SV_ERR_RANGE;
    const CodecLayout L = codec_layout(c);
    if (cap < L.p_off) return SV_ERR_ARG;
    uint32_t* d_sparse = nullptr;
    unsigned long long* d_bsq = nullptr;
    ChunkOut* d_co = nullptr;
    int* d_err = nullptr;
    uint8_t* d_tmp = nullptr;
    unsigned long long* d_mbits = nullptr;
    int32_t* d_kc = nullptr;
    cudaError_t e;
    int r = SV_OK;
    // the encoder writes a whole worst-case slot; use a temporary when cap is smaller
    const bool direct = cap >= L.max_bytes;
    if ((e = cudaMalloc(&d_sparse, (size_t)L.nb * 1024)) || (e = cudaMalloc(&d_bsq, 8ull * L.bpc)) ||
        (e = cudaMalloc(&d_co, sizeof(ChunkOut))) || (e = cudaMalloc(&d_err, sizeof(int))) ||
        (!direct && (e = cudaMalloc(&d_tmp, L.max_bytes))) ||
        (relative && ((e = cudaMalloc(&d_mbits, sizeof(unsigned long long))) ||
                      (e = cudaMalloc(&d_kc, sizeof(int32_t)))))) {
        cudaGetLastError();
        r = SV_ERR_DEVICE_OOM;
    } else {
        uint8_t* dst = direct ? static_cast<uint8_t*>(d_stream) : d_tmp;
        ChunkOut co{};
        int herr = 0;
        cudaMemset(d_err, 0, sizeof(int));
        e = cudaSuccess;
        if (relative)
            e = dtype == SV_C64 ? launch_chunk_steps<float>(d_amps, c, 1, eb, d_mbits, d_kc, 0, nullptr)
                                : launch_chunk_steps<double>(d_amps, c, 1, eb, d_mbits, d_kc, 0, nullptr);
        if (!e)
            e = dtype == SV_C64 ? launch_encode<float>(d_amps, c, dtype, k, 1, dst, L.max_bytes, d_sparse, d_bsq,
                                                       d_co, d_err, 0, nullptr, d_kc)
                                : launch_encode<double>(d_amps, c, dtype, k, 1, dst, L.max_bytes, d_sparse, d_bsq,
                                                        d_co, d_err, 0, nullptr, d_kc);
        if (e || (e = cudaMemcpy(&co, d_co, sizeof(co), cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost))) {
            r = SV_ERR_CUDA;
        } else if (herr & kErrRange) {
            r = SV_ERR_RANGE;
        } else if (co.bytes > cap) {
            r = SV_ERR_ARG;
        } else {
            if (!direct && (e = cudaMemcpy(d_stream, d_tmp, co.bytes, cudaMemcpyDeviceToDevice))) r = SV_ERR_CUDA;
            *h_nbytes = co.bytes;
        }
    }
    cudaFree(d_sparse);
    cudaFree(d_bsq);
    cudaFree(d_co);
    cudaFree(d_err);
    cudaFree(d_tmp);
    cudaFree(d_mbits);
    cudaFree(d_kc);
    return r;
}

int sv_codec_encode(int dtype, int c, double eb, const void* d_amps, void* d_stream, size_t cap, size_t* h_nbytes)
{
    return codec_encode_impl(dtype, c, eb, d_amps, d_stream, cap, h_nbytes, false);
}

int sv_codec_encode_relative(int dtype, int c, double eb, const void* d_amps, void* d_stream, size_t cap,
                             size_t* h_nbytes)
{
    return codec_encode_impl(dtype, c, eb, d_amps, d_stream, cap, h_nbytes, true);
}

int sv_codec_decode(int dtype, int c, const void* d_stream, size_t nbytes, void* d_amps)
{
    if ((dtype != SV_C64 && dtype != SV_C128) || c < 8 || c > 30 || !d_stream || !d_amps) return SV_ERR_ARG;
    const CodecLayout L = codec_layout(c);
    if (nbytes > L.max_bytes || nbytes > 0xffffffffull) return SV_ERR_CORRUPT;
    int* d_err = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_err, sizeof(int)))) return SV_ERR_DEVICE_OOM;
    GroupIn gin{};
    gin.bytes[0] = (uint32_t)nbytes;
    int herr = 0, r = SV_OK;
    cudaMemset(d_err, 0, sizeof(int));
    e = dtype == SV_C64
            ? launch_decode<float>(static_cast<const uint8_t*>(d_stream), L.max_bytes, c, dtype, 1, gin, d_amps, 1.0,
                                   d_err, 0)
            : launch_decode<double>(static_cast<const uint8_t*>(d_stream), L.max_bytes, c, dtype, 1, gin, d_amps, 1.0,
                                    d_err, 0);
    if (e || (e = cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost))) r = SV_ERR_CUDA;
    else if (herr & kErrCorrupt) r = SV_ERR_CORRUPT;
    cudaFree(d_err);
    return r;
}

}  // extern "C"
