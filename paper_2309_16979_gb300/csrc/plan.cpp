// plan.cpp -- circuit partitioning for the compressed state-vector method.
//
// MEMQSim (Sec. 2, "Offline stage") partitions the input circuit into stages
// and the state vector into independently compressed chunks; the online stage
// sweeps all chunks once per stage. The paper gives no partitioning
// algorithm. Here a stage ("pass") is a set of gates whose mixing qubits --
// the targets of non-diagonal gates -- lie in the c low (intra-chunk) qubits
// plus at most g_max staged high qubits S; diagonal gates and controls never
// mix, so they fit any pass. Inside a pass, the same greedy rule splits the
// gates into tile sub-passes whose mixing qubits fit one on-chip tile.
#include <algorithm>
#include <future>
#include <string>
#include <unordered_map>
#include <mutex>
#include <cmath>

#include "runtime.h"

namespace sv {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

bool kind_is_diag(int kind)
{
    switch (kind) {
        case SV_GATE_Z: case SV_GATE_S: case SV_GATE_SDG: case SV_GATE_T: case SV_GATE_TDG:
        case SV_GATE_RZ: case SV_GATE_P: case SV_GATE_CZ: case SV_GATE_CP:
            return true;
        default:
            return false;
    }
}

void gate_matrix(int kind, double theta, const double* custom, int nt, cd* m)
{
    const double r2 = 1.0 / std::sqrt(2.0);
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    const cd I(0, 1);
    for (int i = 0; i < 16; i++) m[i] = 0;
    switch (kind) {
        case SV_GATE_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
        case SV_GATE_X: case SV_GATE_CNOT: m[1] = 1; m[2] = 1; break;
        case SV_GATE_Y: m[1] = -I; m[2] = I; break;
        case SV_GATE_Z: case SV_GATE_CZ: m[0] = 1; m[3] = -1; break;
        case SV_GATE_S: m[0] = 1; m[3] = I; break;
        case SV_GATE_SDG: m[0] = 1; m[3] = -I; break;
        case SV_GATE_T: m[0] = 1; m[3] = cd(r2, r2); break;
        case SV_GATE_TDG: m[0] = 1; m[3] = cd(r2, -r2); break;
        case SV_GATE_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
        case SV_GATE_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
        case SV_GATE_RZ: m[0] = cd(c, -s); m[3] = cd(c, s); break;
        case SV_GATE_P: case SV_GATE_CP: m[0] = 1; m[3] = cd(std::cos(theta), std::sin(theta)); break;
        case SV_GATE_SWAP: m[0] = 1; m[6] = 1; m[9] = 1; m[15] = 1; break;
        case SV_GATE_CUSTOM: {
            const int K = 1 << nt;
            for (int i = 0; i < K * K; i++) m[i] = cd(custom[2 * i], custom[2 * i + 1]);
            break;
        }
        default: break;
    }
}

static uint64_t qubit_mask(const PGate& g)
{
    uint64_t m = 0;
    for (int i = 0; i < g.nt; i++) m |= 1ull << g.t[i];
    for (int i = 0; i < g.nc; i++) m |= 1ull << g.c[i];
    return m;
}

// Qubits a pass must stage for gate g: the targets it mixes, and the target of
// a parameterised gate of a gradient even when it is diagonal (the reverse
// sweep evaluates its generator's partial on the tile, as a register bit).
static uint64_t mixing_mask(const PGate& g)
{
    if (g.diag && g.param < 0) return 0;
    uint64_t m = 0;
    for (int i = 0; i < g.nt; i++) m |= 1ull << g.t[i];
    return m;
}

// A 2x2 matrix commutes with Z when it is diagonal and with X when it is
// symmetric under exchanging its basis states (a I + b X). Exact tests: a
// matrix that misses them by rounding is taken as general.
static bool commutes_z(const cd* m) { return m[1] == cd(0) && m[2] == cd(0); }
static bool commutes_x(const cd* m) { return m[0] == m[3] && m[1] == m[2]; }

// Gates or ops left for later (deferred) block a following one only where
// they do not commute with it: it may run ahead of deferred ones when on
// every qubit it shares with them, it and all of them commute with Z there,
// or it and all of them commute with X there. (Two operators that both
// commute with Z, or both with X, on each qubit they share are sums of
// projectors on those qubits times operators on disjoint qubits, so they
// commute.) A pass's global qubits are controls or diagonal sources only,
// so in the sub-pass and phase planners they never block.
struct Blocked {
    uint64_t any = 0;  // local positions some deferred op touches
    uint64_t nz = 0;   // ... where some deferred op does not commute with Z
    uint64_t nx = 0;   // ... where some deferred op does not commute with X
    bool commute = true;  // false: any shared qubit blocks
    // q: the qubits an op touches; z, x: where it commutes with Z / X
    bool blocks(uint64_t q, uint64_t z, uint64_t x) const
    {
        return (q & any & (commute ? ~((z & ~nz) | (x & ~nx)) : ~0ull)) != 0;
    }
    void add(uint64_t q, uint64_t z, uint64_t x)
    {
        any |= q;
        nz |= q & ~z;
        nx |= q & ~x;
    }
    bool blocks(const HOp& o) const { return blocks(o.qL, o.zL, o.xL); }
    void add(const HOp& o) { add(o.qL, o.zL, o.xL); }
    bool all(uint64_t allL) const { return ((commute ? nz & nx : any) & allL) == allL; }
};

// Qubits where gate g commutes with Z / with X: controls and diagonal
// targets with Z; a single dense target as its matrix does, or, for a
// parameterised gate, as its generator does at every angle (RX: X; RY:
// neither), since a gradient needs the order to hold at all angles.
static void commute_masks(const PGate& g, uint64_t& zm, uint64_t& xm)
{
    zm = xm = 0;
    for (int i = 0; i < g.nc; i++) zm |= 1ull << g.c[i];
    if (g.diag) {
        for (int i = 0; i < g.nt; i++) zm |= 1ull << g.t[i];
        return;
    }
    if (g.nt != 1) return;
    const uint64_t b = 1ull << g.t[0];
    if (g.param >= 0) {
        if (g.kind == SV_GATE_RX) xm |= b;
        return;
    }
    if (commutes_z(g.m)) zm |= b;
    if (commutes_x(g.m)) xm |= b;
}

// Gates one pass staging the high qubits S would apply, scanning the remaining
// gates in order; a gate that cannot run blocks its qubits for later ones.
static int count_pass(const std::vector<PGate>& g, const std::vector<int>& remaining, uint64_t S, uint64_t high,
                      uint64_t all)
{
    Blocked bk;
    int k = 0;
    for (int gi : remaining) {
        const uint64_t qm = qubit_mask(g[gi]);
        uint64_t zm, xm;
        commute_masks(g[gi], zm, xm);
        if (bk.blocks(qm, zm, xm) || (mixing_mask(g[gi]) & high & ~S)) {
            bk.add(qm, zm, xm);
            if (bk.all(all)) break;
            continue;
        }
        k++;
    }
    return k;
}

// One pass over `remaining` (indices into g, in order): the staged set and
// the gates it applies; the gates it leaves, in order, go to `deferred`.
static PassPlan plan_one_pass(const std::vector<PGate>& g, const std::vector<int>& remaining, int n, int c, int gsz,
                              std::vector<int>& deferred)
{
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const uint64_t high = (n > c) ? (all & ~((1ull << c) - 1)) : 0;
    uint64_t S = 0;
    Blocked bk;
    // Stage one high qubit at a time, the one that lets the pass apply the
    // most gates; when none adds any, the scan below stages first-come.
    for (int cur = count_pass(g, remaining, S, high, all); popc(S) < gsz;) {
        int best = -1, bestn = cur;
        for (int q = c; q < n; q++) {
            if ((S >> q) & 1) continue;
            const int k = count_pass(g, remaining, S | (1ull << q), high, all);
            if (k > bestn) {
                bestn = k;
                best = q;
            }
        }
        if (best < 0) break;
        S |= 1ull << best;
        cur = bestn;
    }
    PassPlan pp;
    deferred.clear();
    for (int gi : remaining) {
        const uint64_t qm = qubit_mask(g[gi]);
        uint64_t zm, xm;
        commute_masks(g[gi], zm, xm);
        if (bk.blocks(qm, zm, xm)) {
            deferred.push_back(gi);
            bk.add(qm, zm, xm);
            continue;
        }
        const uint64_t need = mixing_mask(g[gi]) & high & ~S;
        if (popc(S | need) <= gsz) {
            S |= need;
            pp.gates.push_back(gi);
        } else {
            deferred.push_back(gi);
            bk.add(qm, zm, xm);
        }
    }
    // stage exactly gsz high qubits: pad with the lowest unused ones
    for (int q = c; q < n && popc(S) < gsz; q++) S |= 1ull << q;
    for (int q = c; q < n; q++)
        if ((S >> q) & 1) pp.S.push_back(q);
    return pp;
}

std::vector<PassPlan> plan_passes(const std::vector<PGate>& g, int n, int c, int gmax)
{
    std::vector<PassPlan> passes;
    const int gsz = std::min(gmax, n - c);
    std::vector<int> remaining(g.size()), deferred;
    for (size_t i = 0; i < g.size(); i++) remaining[i] = (int)i;
    while (!remaining.empty()) {
        passes.push_back(plan_one_pass(g, remaining, n, c, gsz, deferred));
        remaining.swap(deferred);
    }
    return passes;
}

std::vector<PassPlan> plan_passes_remap(const std::vector<PGate>& g, int n, int c, int gmax, std::vector<PGate>& out,
                                        std::vector<int>& where, std::vector<int>* src)
{
    std::vector<PassPlan> passes;
    const int gsz = std::min(gmax, n - c);
    std::vector<PGate> w = g;       // the gates on the current positions
    std::vector<int> pos(n), at(n);  // pos[q]: position of input qubit q; at[p]: the input qubit at p
    for (int q = 0; q < n; q++) pos[q] = at[q] = q;
    std::vector<int> remaining(g.size()), deferred;
    for (size_t i = 0; i < g.size(); i++) remaining[i] = (int)i;
    out.clear();
    if (src) src->clear();
    constexpr size_t kNever = ~(size_t)0;
    while (!remaining.empty()) {
        PassPlan pp = plan_one_pass(w, remaining, n, c, gsz, deferred);
        std::vector<int> ids;
        for (int gi : pp.gates) {
            ids.push_back((int)out.size());
            out.push_back(w[gi]);
            if (src) src->push_back(gi);
        }
        if (!deferred.empty()) {
            // next[p]: the first of the gates still to run that mixes position p
            std::vector<size_t> next(n, kNever);
            for (size_t k = deferred.size(); k-- > 0;) {
                const uint64_t mm = mixing_mask(w[deferred[k]]);
                for (int p = 0; p < n; p++)
                    if ((mm >> p) & 1) next[p] = k;
            }
            // The low positions and the staged ones hold, after this pass,
            // the qubits mixed soonest (furthest-next-use replacement): pair
            // the staged position needed soonest with the low one needed
            // last while the staged one is needed earlier.
            std::vector<int> hs = pp.S, ls;
            for (int p = 0; p < c; p++) ls.push_back(p);
            std::stable_sort(hs.begin(), hs.end(), [&](int a, int b) { return next[a] < next[b]; });
            std::stable_sort(ls.begin(), ls.end(), [&](int a, int b) { return next[a] > next[b]; });
            int swapped[2][64], ns = 0;
            for (size_t k = 0; k < hs.size() && k < ls.size(); k++) {
                const int h = hs[k], l = ls[k];
                if (next[h] == kNever || next[h] >= next[l]) break;
                PGate sw;
                sw.kind = SV_GATE_SWAP;
                sw.nt = 2;
                sw.t[0] = l;
                sw.t[1] = h;
                gate_matrix(SV_GATE_SWAP, 0, nullptr, 2, sw.m);
                ids.push_back((int)out.size());
                out.push_back(sw);
                if (src) src->push_back(-1);
                swapped[0][ns] = l;
                swapped[1][ns++] = h;
            }
            if (ns) {
                std::vector<int> to(n);  // old position -> new position
                for (int p = 0; p < n; p++) to[p] = p;
                for (int k = 0; k < ns; k++) std::swap(to[swapped[0][k]], to[swapped[1][k]]);
                for (int gi : deferred) {
                    for (int j = 0; j < w[gi].nt; j++) w[gi].t[j] = to[w[gi].t[j]];
                    for (int j = 0; j < w[gi].nc; j++) w[gi].c[j] = to[w[gi].c[j]];
                }
                for (int k = 0; k < ns; k++) {
                    const int a = swapped[0][k], b = swapped[1][k];
                    std::swap(at[a], at[b]);
                    pos[at[a]] = a;
                    pos[at[b]] = b;
                }
            }
        }
        pp.gates = ids;
        passes.push_back(std::move(pp));
        remaining.swap(deferred);
    }
    where = pos;
    return passes;
}

std::vector<PassPlan> plan_circuit(const std::vector<PGate>& g, int n, int c, int gmax, bool remap,
                                   std::vector<PGate>& out, std::vector<int>& where, std::vector<int>* src)
{
    std::vector<PassPlan> passes = plan_passes(g, n, c, gmax);
    out = g;
    where.resize(n);
    for (int q = 0; q < n; q++) where[q] = q;
    if (src) {
        src->resize(g.size());
        for (size_t i = 0; i < g.size(); i++) (*src)[i] = (int)i;
    }
    if (!remap || passes.size() < 2) return passes;
    std::vector<PGate> rg;
    std::vector<int> rw, rs;
    std::vector<PassPlan> rp = plan_passes_remap(g, n, c, gmax, rg, rw, &rs);
    if (rp.size() >= passes.size()) return passes;
    out.swap(rg);
    where.swap(rw);
    if (src) src->swap(rs);
    return rp;
}

std::vector<HOp> local_ops(const std::vector<PGate>& g, const std::vector<int>& ids, int c,
                           const std::vector<int>& S, bool adjoint)
{
    auto loc = [&](int q) -> int {
        if (q < c) return q;
        for (size_t j = 0; j < S.size(); j++)
            if (S[j] == q) return c + (int)j;
        return -1;
    };
    std::vector<HOp> out;
    out.reserve(ids.size());
    for (int gi : ids) {
        const PGate& G = g[gi];
        HOp op;
        for (int i = 0; i < G.nc; i++) {
            const int p = loc(G.c[i]);
            if (p >= 0) { op.cL |= 1ull << p; op.qL |= 1ull << p; op.zL |= 1ull << p; }
            else { op.cG |= 1ull << G.c[i]; op.qG |= 1ull << G.c[i]; }
        }
        if (G.diag) {
            op.type = OP_DIAG;
            for (int i = 0; i < G.nt; i++) {
                const int p = loc(G.t[i]);
                op.dsrc[i] = p >= 0 ? p : kGlobalSrc + G.t[i];
                if (p >= 0) { op.qL |= 1ull << p; op.zL |= 1ull << p; }
                else op.qG |= 1ull << G.t[i];
            }
            const int K = 1 << G.nt;
            for (int v = 0; v < 4; v++) op.m[v] = (v < K) ? G.m[v * K + v] : cd(1, 0);
            if (G.nt == 1) { op.m[2] = op.m[0]; op.m[3] = op.m[1]; }
        } else {
            op.type = G.nt == 1 ? OP_DENSE1 : OP_DENSE2;
            for (int i = 0; i < G.nt; i++) {
                const int p = loc(G.t[i]);
                op.t[i] = p;  // mixing targets are always local in a valid pass
                op.qL |= 1ull << p;
                op.mixL |= 1ull << p;
            }
            for (int i = 0; i < 16; i++) op.m[i] = G.m[i];
            if (G.nt == 1) {
                if (commutes_z(op.m)) op.zL |= op.mixL;
                if (commutes_x(op.m)) op.xL |= op.mixL;
            }
        }
        if (adjoint && G.param >= 0) {
            op.param = G.param;
            op.gen = G.kind == SV_GATE_RX ? 1 : G.kind == SV_GATE_RY ? 2 : 3;
            const int p = loc(G.t[0]);  // >= 0: the pass planner stages a parameterised gate's target
            op.mixL |= 1ull << p;  // the generator's pairs must be tile-local
            if (op.type == OP_DIAG) op.t[0] = p;
            // a gradient needs the ordering to hold at every angle: the
            // generator decides (RX: X-like, RZ: diagonal, RY: neither),
            // not the matrix at this angle (RX(0) is also diagonal)
            const uint64_t b = 1ull << p;
            op.zL = (op.zL & ~b) | (op.gen == 3 ? b : 0);
            op.xL = (op.xL & ~b) | (op.gen == 1 ? b : 0);
        }
        out.push_back(op);
    }
    return out;
}

// ---------------------------------------------------------------- fusion
static bool same_controls(const HOp& a, const HOp& b) { return a.cL == b.cL && a.cG == b.cG; }

static void mat2_mul(const cd* b, const cd* a, cd* out)  // out = b * a (2x2)
{
    cd r[4];
    r[0] = b[0] * a[0] + b[1] * a[2];
    r[1] = b[0] * a[1] + b[1] * a[3];
    r[2] = b[2] * a[0] + b[3] * a[2];
    r[3] = b[2] * a[1] + b[3] * a[3];
    for (int i = 0; i < 4; i++) out[i] = r[i];
}

// 1-bit diagonal on a local position
static bool diag1_local(const HOp& o, int& pos)
{
    if (o.type != OP_DIAG || o.dsrc[1] != -1 || o.dsrc[0] < 0 || o.dsrc[0] >= kGlobalSrc) return false;
    pos = o.dsrc[0];
    return true;
}

// Merge b (applied after a) into a when both act on the same single target
// with the same controls; returns false if they cannot be merged.
static bool try_fuse(HOp& a, const HOp& b)
{
    if (a.param >= 0 || b.param >= 0 || !same_controls(a, b)) return false;
    int pa = -1, pb = -1;
    const bool ad = diag1_local(a, pa), bd = diag1_local(b, pb);
    if (a.type == OP_DENSE1) pa = a.t[0];
    if (b.type == OP_DENSE1) pb = b.t[0];
    if ((a.type != OP_DENSE1 && !ad) || (b.type != OP_DENSE1 && !bd) || pa != pb) return false;
    cd A[4], B[4];
    if (ad) { A[0] = a.m[0]; A[1] = 0; A[2] = 0; A[3] = a.m[1]; }
    else for (int i = 0; i < 4; i++) A[i] = a.m[i];
    if (bd) { B[0] = b.m[0]; B[1] = 0; B[2] = 0; B[3] = b.m[1]; }
    else for (int i = 0; i < 4; i++) B[i] = b.m[i];
    cd M[4];
    mat2_mul(B, A, M);
    if (ad && bd) {
        a.m[0] = M[0]; a.m[1] = M[3]; a.m[2] = M[0]; a.m[3] = M[3];
    } else {
        a.type = OP_DENSE1;
        a.t[0] = pa;
        a.dsrc[0] = a.dsrc[1] = -1;
        a.mixL |= 1ull << pa;
        for (int i = 0; i < 4; i++) a.m[i] = M[i];
        const uint64_t bit = 1ull << pa;
        a.zL = (a.zL & ~bit) | (commutes_z(M) ? bit : 0);
        a.xL = (a.xL & ~bit) | (commutes_x(M) ? bit : 0);
    }
    a.qL |= b.qL;
    a.qG |= b.qG;
    return true;
}

// Ops one sweep with tile set T would apply (no growth of T), scanning the
// remaining ops in order; an op that cannot run blocks its qubits for later
// ones. The scan stops once every local qubit is blocked.
static int count_fit(const std::vector<HOp>& ops, const std::vector<int>& remaining, uint64_t T, uint64_t allL,
                     bool commute)
{
    Blocked bk;
    bk.commute = commute;
    int n = 0;
    for (int oi : remaining) {
        const HOp& o = ops[oi];
        if (bk.blocks(o) || (o.mixL & ~T)) {
            bk.add(o);
            if (bk.all(allL)) break;
            continue;
        }
        n++;
    }
    return n;
}

// Qubits worth adding to tile T: the mixing positions, outside T, of the
// first kLookaheadOps remaining ops that T does not admit.
constexpr int kLookaheadOps = 16;
static uint64_t lookahead_candidates(const std::vector<HOp>& ops, const std::vector<int>& remaining, uint64_t T,
                                     uint64_t allL)
{
    uint64_t cand = 0;
    int seen = 0;
    for (int oi : remaining) {
        const uint64_t need = ops[oi].mixL & ~T & allL;
        if (!need) continue;
        cand |= need;
        if (++seen >= kLookaheadOps) break;
    }
    return cand;
}

// One sub-pass plan. Tiles grow one qubit at a time:
//  - lookahead = false: by the qubit that lets the sweep apply the most ops
//    (pairs of qubits when no single one helps);
//  - lookahead = true: by the candidate qubit whose best follow-up qubit
//    admits the most ops (ties broken by the ops the qubit admits alone),
//    which favours a qubit that is only useful together with another.
// When no growth helps, the scan below grows the tile first-come in circuit
// order.
// groups[s][k]: the indices in `ops` of the ops fused into op k of sub-pass s
using FuseGroups = std::vector<std::vector<std::vector<int>>>;

static std::vector<SubPlan> plan_subpasses_rule(const std::vector<HOp>& ops, int L, int t, int l, bool fuse,
                                                int first_l, bool lookahead, bool commute, FuseGroups& groups)
{
    std::vector<SubPlan> subs;
    groups.clear();
    const uint64_t low = (l >= 64) ? ~0ull : ((1ull << l) - 1);
    const int fl = first_l > 0 ? std::min(first_l, t) : l;
    const uint64_t first_low = (fl >= 64) ? ~0ull : ((1ull << fl) - 1);
    const uint64_t allL = (L >= 64) ? ~0ull : ((1ull << L) - 1);
    std::vector<int> remaining(ops.size());
    for (size_t i = 0; i < ops.size(); i++) remaining[i] = (int)i;
    while (!remaining.empty()) {
        uint64_t T = subs.empty() ? first_low : low;
        Blocked bk;
        bk.commute = commute;
        for (int cur = count_fit(ops, remaining, T, allL, commute); popc(T) < t;) {
            if (lookahead) {
                const uint64_t cand = lookahead_candidates(ops, remaining, T, allL);
                int best = -1, best2 = cur, best1 = cur;
                for (int p = 0; p < L; p++) {
                    if (!((cand >> p) & 1)) continue;
                    const uint64_t Tp = T | (1ull << p);
                    const int k1 = count_fit(ops, remaining, Tp, allL, commute);
                    int k2 = k1;
                    if (popc(Tp) < t)
                        for (int q = 0; q < L; q++)
                            if (q != p && ((cand >> q) & 1)) k2 = std::max(k2, count_fit(ops, remaining, Tp | (1ull << q), allL, commute));
                    if (k2 > best2 || (k2 == best2 && k1 > best1)) {
                        best = p;
                        best2 = k2;
                        best1 = k1;
                    }
                }
                if (best < 0) break;
                T |= 1ull << best;
                cur = best1;
                continue;
            }
            int best = -1, bestn = cur;
            for (int p = 0; p < L; p++) {
                if ((T >> p) & 1) continue;
                const int k = count_fit(ops, remaining, T | (1ull << p), allL, commute);
                if (k > bestn) {
                    bestn = k;
                    best = p;
                }
            }
            if (best >= 0) {
                T |= 1ull << best;
                cur = bestn;
                continue;
            }
            // no single qubit helps: the pair that helps most (two-qubit ops
            // with both qubits outside the tile)
            int b0 = -1, b1 = -1;
            for (int p = 0; p < L && popc(T) + 2 <= t; p++) {
                if ((T >> p) & 1) continue;
                for (int q = p + 1; q < L; q++) {
                    if ((T >> q) & 1) continue;
                    const int k = count_fit(ops, remaining, T | (1ull << p) | (1ull << q), allL, commute);
                    if (k > bestn) {
                        bestn = k;
                        b0 = p;
                        b1 = q;
                    }
                }
            }
            if (b0 < 0) break;
            T |= (1ull << b0) | (1ull << b1);
            cur = bestn;
        }
        SubPlan sp;
        std::vector<std::vector<int>> grp;
        std::vector<int> deferred;
        for (int oi : remaining) {
            const HOp& o = ops[oi];
            if (bk.blocks(o)) {
                deferred.push_back(oi);
                bk.add(o);
                continue;
            }
            const uint64_t need = o.mixL & ~T;
            if (popc(T | need) <= t) {
                T |= need;
                if (fuse && !sp.ops.empty() && try_fuse(sp.ops.back(), o)) {
                    grp.back().push_back(oi);
                    continue;
                }
                sp.ops.push_back(o);
                grp.push_back({oi});
            } else {
                deferred.push_back(oi);
                bk.add(o);
            }
        }
        if (sp.ops.empty() && !deferred.empty() && deferred.size() == remaining.size()) {
            // no op fits a tile (cannot happen when t - l >= 2): stop instead of looping
            subs.clear();
            groups.clear();
            return subs;
        }
        for (int p = 0; p < L && popc(T) < t; p++) T |= 1ull << p;
        sp.T = T;
        subs.push_back(std::move(sp));
        groups.push_back(std::move(grp));
        remaining.swap(deferred);
    }
    return subs;
}

// Plans depend on the ops' structure only (kinds, positions, controls, what
// they touch, whether they carry a parameter), never on their matrices, so
// a process-wide cache keyed by that structure replays a plan for a circuit
// seen before -- the same circuit re-applied, or new angles -- by fusing the
// current ops' matrices along the cached groups. Bounded: cleared when full.
namespace {
struct PlanRecipe {
    std::vector<uint64_t> T;
    FuseGroups groups;
};
std::mutex g_plan_mu;
std::unordered_map<std::string, PlanRecipe> g_plan_cache;
constexpr size_t kPlanCacheMax = 512;

std::string plan_key(const std::vector<HOp>& ops, int L, int t, int l, bool fuse, int first_l)
{
    std::string k;
    k.reserve(20 + ops.size() * 80);
    auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    const int32_t hdr[5] = {L, t, l, fuse ? 1 : 0, first_l};
    put(hdr, sizeof(hdr));
    for (const HOp& o : ops) {
        const int32_t a[6] = {o.type, o.t[0], o.t[1], o.dsrc[0], o.dsrc[1], o.param >= 0 ? 1 : 0};
        const uint64_t b[7] = {o.cL, o.cG, o.qL, o.qG, o.mixL, o.zL, o.xL};
        put(a, sizeof(a));
        put(b, sizeof(b));
    }
    return k;
}

bool replay(const std::vector<HOp>& ops, const PlanRecipe& rc, std::vector<SubPlan>& subs)
{
    subs.clear();
    for (size_t s = 0; s < rc.T.size(); s++) {
        SubPlan sp;
        sp.T = rc.T[s];
        for (const std::vector<int>& g : rc.groups[s]) {
            HOp o = ops[g[0]];
            for (size_t k = 1; k < g.size(); k++)
                if (!try_fuse(o, ops[g[k]])) return false;
            sp.ops.push_back(o);
        }
        subs.push_back(std::move(sp));
    }
    return true;
}
}  // namespace

// Both growth rules (the lookahead on a second thread when the op list is
// long enough to repay it); the plan with fewer sub-passes, the plain rule's
// on a tie.
std::vector<SubPlan> plan_subpasses(const std::vector<HOp>& ops, int L, int t, int l, bool fuse, int first_l)
{
    const std::string key = plan_key(ops, L, t, l, fuse, first_l);
    std::vector<SubPlan> subs;
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        auto it = g_plan_cache.find(key);
        if (it != g_plan_cache.end() && replay(ops, it->second, subs)) return subs;
    }
    // rules: (lookahead, commute) = (no, no), (yes, no), (no, yes), (yes, yes)
    FuseGroups gr[4];
    std::vector<SubPlan> pl[4];
    auto run = [&](int i) { return plan_subpasses_rule(ops, L, t, l, fuse, first_l, (i & 1) != 0, (i & 2) != 0, gr[i]); };
    if (ops.size() < 64) {
        pl[0] = run(0);
        if (pl[0].size() > 1)
            for (int i = 1; i < 4; i++) pl[i] = run(i);
    } else {
        std::future<std::vector<SubPlan>> f[3];
        for (int i = 1; i < 4; i++) f[i - 1] = std::async(std::launch::async, run, i);
        pl[0] = run(0);
        for (int i = 1; i < 4; i++) pl[i] = f[i - 1].get();
    }
    int use = 0;
    for (int i = 1; i < 4; i++)
        if (!pl[i].empty() && pl[i].size() < pl[use].size()) use = i;
    PlanRecipe rc;
    for (const SubPlan& sp : pl[use]) rc.T.push_back(sp.T);
    rc.groups = std::move(gr[use]);
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        if (g_plan_cache.size() >= kPlanCacheMax) g_plan_cache.clear();
        g_plan_cache[key] = std::move(rc);
    }
    return pl[use];
}

bool replan_tail(std::vector<SubPlan>& subs, int L, int t, int l, int last_l, bool keep_first)
{
    const uint64_t want = (last_l >= 64) ? ~0ull : ((1ull << last_l) - 1);
    if (subs.empty() || (subs.back().T & want) == want) return !subs.empty();
    const size_t kmax = std::min<size_t>(3, subs.size() - (keep_first ? 1 : 0));
    for (size_t k = 1; k <= kmax; k++) {
        // the last k sub-passes' ops, in the planned order, backwards
        std::vector<HOp> rev;
        for (size_t i = subs.size() - k; i < subs.size(); i++)
            for (const HOp& o : subs[i].ops) rev.push_back(o);
        std::reverse(rev.begin(), rev.end());
        std::vector<SubPlan> alt = plan_subpasses(rev, L, t, l, false, last_l);
        if (alt.empty() || alt.size() > k) continue;
        std::reverse(alt.begin(), alt.end());
        for (SubPlan& sp : alt) {
            std::reverse(sp.ops.begin(), sp.ops.end());
            std::vector<HOp> fused;
            for (const HOp& o : sp.ops)
                if (fused.empty() || !try_fuse(fused.back(), o)) fused.push_back(o);
            sp.ops.swap(fused);
        }
        subs.resize(subs.size() - k);
        for (SubPlan& sp : alt) subs.push_back(std::move(sp));
        return true;
    }
    return false;
}

TileDesc tile_desc(uint64_t T, int L, int t, int l)
{
    TileDesc td{};
    td.t = t;
    td.l = l;
    td.L = L;
    int h = 0, o = 0;
    for (int p = 0; p < L; p++) {
        if ((T >> p) & 1) {
            if (p >= l) td.hpos[h++] = (int8_t)p;
        } else {
            td.opos[o++] = (int8_t)p;
        }
    }
    td.nout = o;
    return td;
}

template <typename R>
void dev_ops(const SubPlan& sp, const TileDesc& td, std::vector<DevOp<R>>& out, int* grad_slot_base,
             std::vector<int>* slot_params)
{
    // local position -> tile bit
    int tpos[64];
    for (int p = 0; p < 64; p++) tpos[p] = -1;
    for (int p = 0; p < td.l; p++) tpos[p] = p;
    for (int i = 0; i < td.t - td.l; i++) tpos[td.hpos[i]] = td.l + i;
    for (const HOp& o : sp.ops) {
        DevOp<R> d{};
        d.type = o.type;
        d.grad_slot = -1;
        d.gen = 0;
        d.d0 = d.d1 = SRC_NONE;
        for (int p = 0; p < 64; p++) {
            if (!((o.cL >> p) & 1)) continue;
            if (tpos[p] >= 0) d.cmask_tile |= 1u << tpos[p];
            else d.cmask_local |= 1ull << p;
        }
        d.cmask_global = o.cG;
        if (o.type == OP_DIAG) {
            int32_t* dst[2] = {&d.d0, &d.d1};
            for (int i = 0; i < 2; i++) {
                const int s = o.dsrc[i];
                if (s < 0) *dst[i] = SRC_NONE;
                else if (s >= kGlobalSrc) *dst[i] = SRC_GLOBAL + (s - kGlobalSrc);
                else if (tpos[s] >= 0) *dst[i] = SRC_TILE + tpos[s];
                else *dst[i] = SRC_LOCAL + s;
            }
            for (int v = 0; v < 4; v++) { d.m[2 * v] = (R)o.m[v].real(); d.m[2 * v + 1] = (R)o.m[v].imag(); }
            if (o.param >= 0) d.t0 = tpos[o.t[0]];
        } else {
            d.t0 = tpos[o.t[0]];
            d.t1 = o.type == OP_DENSE2 ? tpos[o.t[1]] : 0;
            const int K = o.type == OP_DENSE2 ? 4 : 2;
            for (int i = 0; i < K * K; i++) { d.m[2 * i] = (R)o.m[i].real(); d.m[2 * i + 1] = (R)o.m[i].imag(); }
        }
        if (o.param >= 0 && grad_slot_base) {
            d.grad_slot = (*grad_slot_base)++;
            d.gen = o.gen;
            if (slot_params) slot_params->push_back(o.param);
        }
        out.push_back(d);
    }
}

// --------------------------------------------------------- register phases
static int classify_2x2(const cd* m)
{
    bool real = true, rx = true;
    for (int i = 0; i < 4; i++)
        if (m[i].imag() != 0) real = false;
    if (m[0].imag() != 0 || m[3].imag() != 0 || m[1].real() != 0 || m[2].real() != 0) rx = false;
    if (real) return PK_REAL;
    if (rx) return PK_RX;
    return PK_GENERIC;
}

// The register sets and op placement of a sub-pass's phases depend on its
// ops' structure and the tile's numbering only, not on their matrices; the
// enumerated plan costs a few hundred placements per phase, so a
// process-wide cache (bounded, cleared when full) keeps them per structure.
namespace {
struct PhasePick {
    uint32_t Rm;
    std::vector<int> placed;
};
std::mutex g_phase_mu;
std::unordered_map<std::string, std::vector<PhasePick>> g_phase_cache;
constexpr size_t kPhaseCacheMax = 4096;

std::string phase_key(const SubPlan& sp, const TileDesc& td, bool adjoint)
{
    std::string k;
    k.reserve(16 + sp.ops.size() * 32);
    auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    const int32_t hdr[3] = {td.t, td.l, adjoint ? 1 : 0};
    put(hdr, sizeof(hdr));
    put(td.hpos, (size_t)(td.t - td.l));
    for (const HOp& o : sp.ops) {
        const uint64_t b[4] = {o.qL, o.mixL, o.zL, o.xL};
        put(b, sizeof(b));
    }
    return k;
}
}  // namespace

template <typename R>
void dev_phases(const SubPlan& sp, const TileDesc& td, std::vector<Phase>& phases, std::vector<PhaseOp<R>>& out,
                std::vector<CtaCtrl>& ctl, std::vector<R>& d2m, std::vector<int32_t>* grad,
                std::vector<int>* slot_params)
{
    int nslot = 0;
    int tbit[64];  // local position -> tile bit (-1 outside the tile)
    for (int p = 0; p < 64; p++) tbit[p] = -1;
    for (int p = 0; p < td.l; p++) tbit[p] = p;
    for (int i = 0; i < td.t - td.l; i++) tbit[td.hpos[i]] = td.l + i;
    const int nops = (int)sp.ops.size();
    std::vector<uint32_t> mix(nops, 0);
    for (int i = 0; i < nops; i++) {
        const HOp& o = sp.ops[i];
        for (int p = 0; p < 64; p++)
            if ((o.mixL >> p) & 1) mix[i] |= 1u << tbit[p];
    }
    // ops a phase with register bits `regs` applies, in order: those whose
    // mixing bits lie in regs and that no deferred op before them blocks
    auto place_with = [&](const std::vector<int>& rem, uint32_t regs, std::vector<int>* placed,
                          std::vector<int>* deferred) {
        Blocked bk;
        int n = 0;
        for (int oi : rem) {
            const HOp& o = sp.ops[oi];
            if (bk.blocks(o) || (mix[oi] & ~regs)) {
                if (deferred) deferred->push_back(oi);
                bk.add(o);
                continue;
            }
            if (placed) placed->push_back(oi);
            n++;
        }
        return n;
    };
    // The phases' register bits and ops. First-come: ops in order while their
    // mixing bits fit kPhaseRegBits. Enumerated: per phase, the set of
    // kPhaseRegBits of the remaining ops' bits that applies the most ops (the
    // first-come set reproduces itself under place_with, so it is among the
    // candidates and wins ties).
    auto plan_phases = [&](bool enumerate) {
        std::vector<PhasePick> out;
        std::vector<int> remaining(nops);
        for (int i = 0; i < nops; i++) remaining[i] = i;
        while (!remaining.empty()) {
            uint32_t Rm = 0;
            Blocked bk;
            std::vector<int> placed, deferred;
            for (int oi : remaining) {
                const HOp& o = sp.ops[oi];
                if (bk.blocks(o)) {
                    deferred.push_back(oi);
                    bk.add(o);
                    continue;
                }
                if (popc(Rm | mix[oi]) <= kPhaseRegBits) {
                    Rm |= mix[oi];
                    placed.push_back(oi);
                } else {
                    deferred.push_back(oi);
                    bk.add(o);
                }
            }
            uint32_t U = 0;
            for (int oi : remaining) U |= mix[oi];
            if (enumerate && popc(U) > kPhaseRegBits) {
                int best = (int)placed.size();
                uint32_t bestR = 0;
                // candidates in local-position order, so that the pick (ties
                // included) does not depend on how the tile numbers its high bits
                std::vector<int> ub;
                for (int p = 0; p < 64; p++)
                    if (tbit[p] >= 0 && ((U >> tbit[p]) & 1)) ub.push_back(tbit[p]);
                const int m = (int)ub.size();
                for (int a = 0; a < m; a++)
                    for (int b = a + 1; b < m; b++)
                        for (int c2 = b + 1; c2 < m; c2++)
                            for (int d = c2 + 1; d < m; d++) {
                                const uint32_t regs = (1u << ub[a]) | (1u << ub[b]) | (1u << ub[c2]) | (1u << ub[d]);
                                const int k = place_with(remaining, regs, nullptr, nullptr);
                                if (k > best) {
                                    best = k;
                                    bestR = regs;
                                }
                            }
                if (bestR) {
                    placed.clear();
                    deferred.clear();
                    place_with(remaining, bestR, &placed, &deferred);
                    Rm = bestR;
                }
            }
            // unused register bits: the lowest tile bits, except in the last phase,
            // which leaves tile bits 0..3 to thread bits 0..3 (its stores can then
            // go from registers straight to HBM in whole 32-byte sectors) and takes
            // the tile's highest local positions, again whatever their numbering
            if (deferred.empty()) {
                for (int p = 63; p >= 0 && popc(Rm) < kPhaseRegBits; p--)
                    if (tbit[p] >= 0) Rm |= 1u << tbit[p];
            } else {
                for (int b = 0; b < td.t && popc(Rm) < kPhaseRegBits; b++) Rm |= 1u << b;
            }
            out.push_back({Rm, std::move(placed)});
            remaining.swap(deferred);
        }
        return out;
    };
    // Forward sub-passes take the enumerated phases when they cost less,
    // counting one shared-memory round trip per phase and one more for a last
    // phase that cannot store straight to HBM (tile bits 0 and 1 in its
    // registers). Adjoint sub-passes keep first-come (measured slower with the
    // larger phases: their gradient partials sit between the ops).
    const std::string key = phase_key(sp, td, grad != nullptr);
    std::vector<PhasePick> picks;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_phase_mu);
        auto it = g_phase_cache.find(key);
        if (it != g_phase_cache.end()) {
            picks = it->second;
            cached = true;
        }
    }
    if (!cached) {
        picks = plan_phases(false);
        if (!grad) {
            std::vector<PhasePick> alt = plan_phases(true);
            auto cost = [](const std::vector<PhasePick>& v) {
                return v.size() + (v.empty() || (v.back().Rm & 3u) ? 1 : 0);
            };
            if (cost(alt) < cost(picks)) picks.swap(alt);
        }
        std::lock_guard<std::mutex> lock(g_phase_mu);
        if (g_phase_cache.size() >= kPhaseCacheMax) g_phase_cache.clear();
        g_phase_cache[key] = picks;
    }
    for (const PhasePick& pick : picks) {
        const uint32_t Rm = pick.Rm;
        const std::vector<int>& placed = pick.placed;
        Phase ph{};
        int reg_of[32];
        for (int b = 0; b < 32; b++) reg_of[b] = -1;
        int j = 0;
        for (int b = 0; b < td.t; b++)
            if ((Rm >> b) & 1) { ph.rpos[j] = (int8_t)b; reg_of[b] = j++; }
        // thread bits 0..3 on tile bits of distinct residues mod 4 (bank spread), then the rest
        bool used[32] = {};
        int k = 0;
        for (int r = 0; r < 4; r++)
            for (int b = r; b < td.t; b += 4)
                if (!((Rm >> b) & 1) && !used[b]) { ph.tpos[k++] = (int8_t)b; used[b] = true; break; }
        for (int b = 0; b < td.t; b++)
            if (!((Rm >> b) & 1) && !used[b]) { ph.tpos[k++] = (int8_t)b; used[b] = true; }
        ph.op_begin = (int)out.size();
        // constant bit source byte of a local position / global qubit (see kSrcNone)
        auto csrc_of = [&](int s) -> uint8_t {
            if (s < 0) return kSrcNone;
            if (s >= kGlobalSrc) return (uint8_t)(0x80 + (s - kGlobalSrc));
            if (tbit[s] < 0) return (uint8_t)(0x40 + s);
            return (uint8_t)tbit[s];
        };
        for (int oi : placed) {
            const HOp& o = sp.ops[oi];
            PhaseOp<R> d{};
            d.csrc = d.csrc1 = kSrcNone;
            uint32_t creg = 0;
            CtaCtrl cc{0, 0};
            for (int p = 0; p < 64; p++) {
                if (!((o.cL >> p) & 1)) continue;
                const int b = tbit[p];
                if (b < 0) cc.cl |= 1ull << p;
                else if (reg_of[b] >= 0) creg |= 1u << reg_of[b];
                else d.tmask |= (uint16_t)(1u << b);
            }
            cc.cg = o.cG;
            if (cc.cl || cc.cg) {
                d.flags = 1;
                d.aux = (uint32_t)ctl.size();
                ctl.push_back(cc);
            }
            uint32_t kind, b0 = 0, b1 = 0, excl = 0;
            if (o.type == OP_DIAG) {
                const int s0 = o.dsrc[0], s1 = o.dsrc[1];
                const int r0 = (s0 >= 0 && s0 < kGlobalSrc && tbit[s0] >= 0) ? reg_of[tbit[s0]] : -1;
                const int r1 = (s1 >= 0 && s1 < kGlobalSrc && tbit[s1] >= 0) ? reg_of[tbit[s1]] : -1;
                if (r0 >= 0 && r1 >= 0) {
                    kind = PK_DIAG2; b0 = r0; b1 = r1;
                } else if (r0 >= 0 || r1 >= 0) {
                    kind = PK_DIAG1;
                    b0 = r0 >= 0 ? r0 : r1;
                    d.rsel = r0 >= 0 ? 0 : 1;
                    d.csrc = csrc_of(r0 >= 0 ? s1 : s0);
                } else {
                    kind = PK_DIAGT;
                    d.csrc = csrc_of(s0);
                    d.csrc1 = csrc_of(s1);
                }
                for (int v = 0; v < 4; v++) { d.m[2 * v] = (R)o.m[v].real(); d.m[2 * v + 1] = (R)o.m[v].imag(); }
            } else if (o.type == OP_DENSE1) {
                kind = (uint32_t)classify_2x2(o.m);
                b0 = reg_of[tbit[o.t[0]]];
                excl = 1u << b0;  // pairs are enumerated from their b0 = 0 member
                for (int i = 0; i < 4; i++) { d.m[2 * i] = (R)o.m[i].real(); d.m[2 * i + 1] = (R)o.m[i].imag(); }
            } else {
                kind = PK_DENSE2;
                b0 = reg_of[tbit[o.t[0]]];
                b1 = reg_of[tbit[o.t[1]]];
                excl = (1u << b0) | (1u << b1);
                d.aux = (uint32_t)(d2m.size() / 32);
                for (int i = 0; i < 16; i++) { d2m.push_back((R)o.m[i].real()); d2m.push_back((R)o.m[i].imag()); }
            }
            // register indices that take part: every control bit set (pair/quad leaders only for dense ops)
            uint32_t am = 0;
            for (uint32_t i = 0; i < 16; i++)
                if (!(i & excl) && (i & creg) == creg) am |= 1u << i;
            d.amask = (uint16_t)am;
            const uint32_t ctrl = creg != 0 ? 1u : 0u;
            if (kind <= PK_DIAG1) d.code = (uint16_t)(kind * 8 + ctrl * 4 + b0);
            else if (kind == PK_DIAG2) d.code = (uint16_t)(kCodeDiag2 + ctrl * 16 + b1 * 4 + b0);
            else if (kind == PK_DIAGT) d.code = (uint16_t)(kCodeDiagT + ctrl);
            else {
                d.code = (uint16_t)kCodeDense2;
                d.pad = (uint16_t)(b1 * 4 + b0);
            }
            out.push_back(d);
            if (grad) {
                if (o.param >= 0) {
                    grad->push_back((nslot++ << 2) | o.gen);
                    if (slot_params) slot_params->push_back(o.param);
                } else {
                    grad->push_back(-1);
                }
            }
        }
        // swizzled shared-memory offset of each register index (the swizzle is
        // linear over XOR, so the device adds the thread's part with one XOR)
        for (int m = 0; m < 16; m++) {
            uint32_t o = 0;
            for (int q = 0; q < kPhaseRegBits; q++)
                if ((m >> q) & 1) o |= 1u << ph.rpos[q];
            ph.sroff[m] = (uint16_t)(o ^ (((o >> 4) ^ (o >> 8)) & 15u));
        }
        ph.op_count = (int)out.size() - ph.op_begin;
        phases.push_back(ph);
    }
}

// Number the tile's high bits so that no register phase holds a whole class
// of tile bits with the same index mod 4. The padded shared-memory layout
// moves tile bit b by 2^(b mod 4) slots mod 16, so a half-warp's 64-bit
// accesses are free of bank conflicts only when its four thread bits cover
// the four classes, and a phase whose register bits include a whole class
// leaves its threads none of that class. Which local qubits a phase holds in
// registers does not depend on the numbering; a deterministic search over
// orders of the high bits keeps the first with the fewest such phases.
template <typename R>
void order_tile_bits(const SubPlan& sp, TileDesc& td, bool adjoint)
{
    const int nh = td.t - td.l;
    if (td.t != kPhaseTileQubits || nh < 2) return;
    std::vector<Phase> ph;
    std::vector<PhaseOp<R>> ops;
    std::vector<CtaCtrl> ctl;
    std::vector<R> d2m;
    std::vector<int32_t> grad;  // the adjoint's phases are planned as its sub-passes' are
    dev_phases<R>(sp, td, ph, ops, ctl, d2m, adjoint ? &grad : nullptr);
    // each phase's register qubits as local positions
    std::vector<uint64_t> reg(ph.size(), 0);
    for (size_t i = 0; i < ph.size(); i++)
        for (int j = 0; j < kPhaseRegBits; j++) {
            const int b = ph[i].rpos[j];
            reg[i] |= 1ull << (b < td.l ? b : td.hpos[b - td.l]);
        }
    auto bad = [&](const int8_t* hp) {
        int n = 0;
        for (uint64_t rl : reg) {
            uint32_t rt = 0;  // tile bits of the phase's registers under numbering hp
            for (int b = 0; b < td.l; b++)
                if ((rl >> b) & 1) rt |= 1u << b;
            for (int i = 0; i < nh; i++)
                if ((rl >> hp[i]) & 1) rt |= 1u << (td.l + i);
            for (int r = 0; r < 4; r++) {
                uint32_t cls = 0;
                for (int b = r; b < td.t; b += 4) cls |= 1u << b;
                if ((rt & cls) == cls) n++;
            }
        }
        return n;
    };
    int best = bad(td.hpos);
    if (best == 0) return;
    int8_t cur[kMaxTileQubits], keep[kMaxTileQubits];
    for (int i = 0; i < nh; i++) cur[i] = keep[i] = td.hpos[i];
    uint64_t x = 0x9e3779b97f4a7c15ull;  // splitmix64 state: the search is deterministic
    for (int trial = 0; trial < 256 && best > 0; trial++) {
        for (int i = nh - 1; i > 0; i--) {
            x += 0x9e3779b97f4a7c15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
            z ^= z >> 31;
            std::swap(cur[i], cur[z % (uint64_t)(i + 1)]);
        }
        const int v = bad(cur);
        if (v < best) {
            best = v;
            for (int i = 0; i < nh; i++) keep[i] = cur[i];
        }
    }
    for (int i = 0; i < nh; i++) td.hpos[i] = keep[i];
}

template void order_tile_bits<float>(const SubPlan&, TileDesc&, bool);
template void order_tile_bits<double>(const SubPlan&, TileDesc&, bool);

template void dev_phases<float>(const SubPlan&, const TileDesc&, std::vector<Phase>&, std::vector<PhaseOp<float>>&,
                                std::vector<CtaCtrl>&, std::vector<float>&, std::vector<int32_t>*, std::vector<int>*);
template void dev_phases<double>(const SubPlan&, const TileDesc&, std::vector<Phase>&, std::vector<PhaseOp<double>>&,
                                 std::vector<CtaCtrl>&, std::vector<double>&, std::vector<int32_t>*,
                                 std::vector<int>*);

template void dev_ops<float>(const SubPlan&, const TileDesc&, std::vector<DevOp<float>>&, int*, std::vector<int>*);
template void dev_ops<double>(const SubPlan&, const TileDesc&, std::vector<DevOp<double>>&, int*,
                              std::vector<int>*);

}  // namespace sv
