// runtime.h -- host runtime of the compressed state-vector simulator: gate
// representation, pass planning, the pinned compressed chunk store and the
// state handle behind the C ABI in include/sv.h.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <map>
#include <vector>

#include "sv.h"
#include "sv_internal.h"

namespace sv {

using cd = std::complex<double>;

// A validated gate on physical qubits (SWAPs already absorbed).
struct PGate {
    int kind = 0;
    int nt = 1, nc = 0;
    int t[2] = {0, 0};
    int c[2] = {0, 0};
    double theta = 0;
    int param = -1;
    bool diag = false;
    cd m[16];
};

// Matrix of a gate kind on its targets (row-major 2^nt x 2^nt, FP64).
void gate_matrix(int kind, double theta, const double* custom, int nt, cd* m);
bool kind_is_diag(int kind);

// Host op in a pass's local coordinates (before tiling).
constexpr int kGlobalSrc = 1000;  // diag source >= kGlobalSrc: global qubit (src - kGlobalSrc)

struct HOp {
    int type = OP_DENSE1;
    int t[2] = {0, 0};             // local positions of dense targets
    int dsrc[2] = {-1, -1};        // diag entry-index bit sources: local position or kGlobalSrc + q
    uint64_t cL = 0, cG = 0;       // controls: local positions / global qubits
    cd m[16];
    int param = -1;                // adjoint: parameter index
    int gen = 0;                   // adjoint: 1 X, 2 Y, 3 Z
    uint64_t qL = 0, qG = 0;       // every qubit the op touches (for ordering)
    uint64_t mixL = 0;             // local positions that must be tile bits
    // local positions where the op commutes with Z (controls, diagonal
    // sources, diagonal targets) / with X (X-like targets: X, RX, CNOT's
    // target); global qubits are only ever controls or diagonal sources
    uint64_t zL = 0, xL = 0;
};

struct SubPlan {
    uint64_t T = 0;                // tile positions (local)
    std::vector<HOp> ops;
};

struct PassPlan {
    std::vector<int> S;            // staged high qubits (physical), ascending
    std::vector<int> gates;        // indices into the physical gate list
    std::vector<SubPlan> subs;
};

// Chunk-level passes: gates in order, each pass holding the gates whose
// mixing high qubits fit in g_max staged qubits; gates are moved ahead only
// past gates on disjoint qubits.
std::vector<PassPlan> plan_passes(const std::vector<PGate>& g, int n, int c, int gmax);

// The same passes with qubit remapping: at the end of each pass, staged high
// positions whose qubits the remaining gates mix before those of some low
// positions exchange qubits with them (a physical SWAP applied in the pass),
// and the gates after it run on the new positions. `out` receives the
// physical gate list the passes index (the input's gates on their new
// positions plus the SWAPs), `where[q]` the final position of the qubit at
// input position q; src (if given) the input index of each entry of `out`,
// -1 for the SWAPs.
std::vector<PassPlan> plan_passes_remap(const std::vector<PGate>& g, int n, int c, int gmax, std::vector<PGate>& out,
                                        std::vector<int>& where, std::vector<int>* src = nullptr);

// The passes a circuit runs as: plan_passes, or with `remap` the remapped
// passes when they are fewer. `out` receives the gate list the passes index,
// `where` the final positions (the identity without remapping), src (if
// given) the input index of each gate of `out` (-1 for an added SWAP).
std::vector<PassPlan> plan_circuit(const std::vector<PGate>& g, int n, int c, int gmax, bool remap,
                                   std::vector<PGate>& out, std::vector<int>& where,
                                   std::vector<int>* src = nullptr);

// Translate a pass's gates to local ops: low qubits 0..c-1 keep their
// position, S[j] becomes position c + j, other qubits are global.
std::vector<HOp> local_ops(const std::vector<PGate>& g, const std::vector<int>& ids, int c,
                           const std::vector<int>& S, bool adjoint);

// Tile sub-passes over L local positions (tiles of t qubits containing 0..l-1).
// first_l > 0: the first sub-pass's tile must contain local bits 0..first_l-1.
std::vector<SubPlan> plan_subpasses(const std::vector<HOp>& ops, int L, int t, int l, bool fuse, int first_l = 0);

// Make the last tile contain local bits 0..last_l-1 without adding a
// sub-pass: the ops of the last k <= 3 sub-passes (a suffix of the planned
// order) are planned again backwards, the first tile of that backward plan
// required to hold the bits (reversing a sequence keeps which ops commute),
// and put back in forward order. keep_first: leave subs[0] unchanged.
// Returns whether the last tile holds the bits.
bool replan_tail(std::vector<SubPlan>& subs, int L, int t, int l, int last_l, bool keep_first);

// Tile descriptor and device ops of one sub-pass.
TileDesc tile_desc(uint64_t T, int L, int t, int l);
// Renumber the high bits of a 2^12 tile against shared-memory bank
// conflicts of its register phases (plan.cpp); adjoint: the phases are
// those of an adjoint sub-pass.
template <typename R>
void order_tile_bits(const SubPlan& sp, TileDesc& td, bool adjoint);
template <typename R>
void dev_ops(const SubPlan& sp, const TileDesc& td, std::vector<DevOp<R>>& out, int* grad_slot_base,
             std::vector<int>* slot_params);

// Register phases of one sub-pass on a 2^12 tile (apply_phase.cu, jit.cpp).
// With `grad` (adjoint sub-passes): one entry per op appended to `out`, -1 or
// (gradient slot << 2) | generator (1 X, 2 Y, 3 Z), slots numbered from 0 in
// the order the ops are placed; slot_params receives each slot's parameter.
template <typename R>
void dev_phases(const SubPlan& sp, const TileDesc& td, std::vector<Phase>& phases, std::vector<PhaseOp<R>>& out,
                std::vector<CtaCtrl>& ctl, std::vector<R>& d2m, std::vector<int32_t>* grad = nullptr,
                std::vector<int>* slot_params = nullptr);

// ------------------------------------------------------------- the store
struct Segment {
    uint8_t* ptr = nullptr;
    size_t cap = 0;
};

// Pinned host memory of a compressed chunk store: slots carved best-fit from
// large pinned segments; a released slot merges with free neighbours of the
// same segment (a slot never spans two pinned allocations).
struct HostPool {
    std::vector<Segment> segs;
    size_t seg_bytes = 0;  // size of a new segment (a smaller one when the host budget is nearly spent)
    std::map<uint8_t*, std::pair<size_t, int>> free_at;  // free block -> (bytes, segment)
    std::multimap<size_t, uint8_t*> free_by_size;
    uint8_t* shared = nullptr;  // the slot chunks share while they hold the same stream (read only)
    size_t shared_cap = 0;
};

// One chunk's stream in the store: `bytes` long in a slot of `cap` bytes.
struct ChunkRef {
    uint8_t* ptr = nullptr;
    uint64_t bytes = 0;
    uint64_t cap = 0;
};

}  // namespace sv

// The opaque handle of the C ABI.
struct sv_state {
    int n = 0, c = 0, dtype = SV_C64, mode = SV_COMPRESSED;
    double eb = 0;
    int k = 0;                      // codec step exponent
    int kl = 0;                     // step exponent of the lambda store (k + ceil(log2 sum|c|))
    sv_config cfg{};
    int gmax = 4, tq = 12, lq = 5, nslots = 3;
    int nh = 0;                     // high qubits n - c
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    // ordering against the caller's stream (sv_config.stream)
    cudaEvent_t ev_user = nullptr, ev_done = nullptr;
    // compressed store and staging
    size_t stride = 0;              // device slot stride per chunk stream
    std::vector<sv::ChunkRef> cur;  // one slot per chunk, rewritten in place by each pass
    sv::HostPool pool;
    uint64_t pinned_bytes = 0;
    uint8_t* d_in[4] = {};
    uint8_t* d_out[4] = {};
    sv::ChunkOut* d_co[4] = {};
    sv::ChunkOut* h_co[4] = {};
    cudaEvent_t ev_h2d[4] = {}, ev_comp[4] = {}, ev_d2h[4] = {};
    bool slot_used[4] = {};
    // Cross-pass pipelining inside one sv_apply_circuit: the streams of the last
    // group of a pass are copied on the device into d_carry (chunk k at
    // carry_at[k] * stride, -1 when not carried) so the next pass starts
    // without their host round trip; ev_prev_d2h is recorded after the latest
    // device -> host copies.
    uint8_t* d_carry = nullptr;
    uint64_t* d_carry_bytes = nullptr;  // lengths of the streams in d_carry
    std::vector<int32_t> carry_at;
    cudaEvent_t ev_prev_d2h = nullptr;
    void* d_amps = nullptr;
    uint32_t* d_sparse = nullptr;
    unsigned long long* d_blocksq = nullptr;
    int* d_err = nullptr;
    // uncompressed state / adjoint vectors
    void* d_state = nullptr;
    void* d_lam = nullptr;
    // compressed adjoint: lambda = H psi as a second compressed chunk store with
    // its own slots and staging (allocated at the first compressed sv_grad)
    std::vector<sv::ChunkRef> lcur;  // the lambda store of sv_grad, one slot per chunk
    sv::HostPool lpool;
    uint8_t* d_in2[4] = {};
    uint8_t* d_out2[4] = {};
    sv::ChunkOut* d_co2[4] = {};
    sv::ChunkOut* h_co2[4] = {};
    void* d_amps2 = nullptr;
    // relative bound: per-chunk step exponents of a group and their scratch
    bool rel = false;
    int32_t* d_kc = nullptr;
    unsigned long long* d_mbits = nullptr;
    // device op list
    void* d_ops = nullptr;
    size_t ops_cap = 0;
    // logical -> physical qubit
    std::vector<int> perm;
    double scale = 1.0;             // decode scale (renormalisation)
    sv_stats_t st{};
    std::string err;
    // profiling: event pairs around kernel launches on s_comp, read at pass end
    struct ProfRec { int kind; uint64_t bytes; };
    std::vector<cudaEvent_t> prof_ev;
    std::vector<ProfRec> prof_rec;
    size_t prof_used = 0;
};
