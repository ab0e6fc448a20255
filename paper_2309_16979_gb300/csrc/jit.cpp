// jit.cpp -- sub-pass kernels specialised to their gate sequence (MEMQSim
// Sec. 2, "Online stage" step (3): the kernel that applies a pass's fused
// gates to the staged chunk group), generated at run time and compiled with
// NVRTC for the device in use.
//
// The table-driven phase kernel (apply_phase.cu) spends most of its issue
// slots interpreting its op stream: fetching each op's record, dispatching on
// its form, reconciling registers between forms. Here each sub-pass becomes a
// kernel of its own, written out as straight-line code: per phase, the
// sixteen register loads at the phase's swizzled offsets, then every gate as
// exactly the multiply-adds its matrix needs, then the stores.
//
// What is baked into the code is the sub-pass's structure: the phases'
// register and thread bits, each gate's target bits and controls, and which
// matrix entries are exactly 0, +-1 or +-i (a zero drops a term, +-1 and +-i
// turn a product into a move or a negation; an X, or any 0/1 permutation
// whose controls are all register bits, only renames the registers holding
// the pair). Every other entry is read from the kernel's by-value parameter
// block (the constant bank), so circuits that differ only in their rotation
// angles share kernels. Kernels are cached per process by their source text.
#include "jit.h"

#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <map>
#include <atomic>
#include <chrono>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <memory>
#include <mutex>
#include <sstream>
#include <thread>
#include <unordered_map>

#include "jit_embed.inc"  // kJitHeaderNames / kJitHeaders / kJitHeaderCount: device headers the kernels include

namespace sv {

struct JitFn {
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    int lrow = 0;  // low bits of the tile rows the kernel was generated for
};

namespace {

constexpr size_t kMaxParamBytes = 24576;  // by-value parameter block cap (CUDA allows 32764 bytes in all)
constexpr int kJitThreads = 256;
constexpr size_t kKeyHeader = 5;  // key bytes: sizeof(R), dec, enc, mode, row bits

// slot of tile offset x in the padded shared-memory layout (tile::PadLayout)
uint32_t pad_slot(uint32_t x) { return x + (x >> 4) + (x >> 8); }
// slots of one padded tile buffer (tile::kPadElems)
size_t tile_pad_elems() { return (pad_slot((1u << kPhaseTileQubits) - 1) + 1 + 15) & ~size_t(15); }

// Complex64 sub-passes that read amplitudes from HBM double-buffer the tile:
// the next tile's copy is in flight while the current one is processed.
bool prefetches(bool dec, size_t rsize) { return rsize == 4 && !dec; }

// ------------------------------------------------------------ generation
// A complex coefficient as the generated code sees it.
enum Cls { C_ZERO, C_ONE, C_MONE, C_I, C_MI, C_REAL, C_IMAG, C_GEN };

struct Coef {
    int cls = C_ZERO;
    std::string re, im;  // expressions of the parts a REAL / IMAG / GEN coefficient reads
};

std::string pref(size_t i) { return "p.m[" + std::to_string(i) + "]"; }

template <typename R>
int entry_class(R re, R im)
{
    if (re == 0 && im == 0) return C_ZERO;
    if (re == 1 && im == 0) return C_ONE;
    if (re == -1 && im == 0) return C_MONE;
    if (re == 0 && im == 1) return C_I;
    if (re == 0 && im == -1) return C_MI;
    if (im == 0) return C_REAL;
    if (re == 0) return C_IMAG;
    return C_GEN;
}

template <typename R>
Coef fixed_coef(R re, R im, size_t pidx)
{
    Coef c;
    c.cls = entry_class(re, im);
    c.re = pref(pidx);
    c.im = pref(pidx + 1);
    return c;
}

// A real sum of signed products, written so that the compiler contracts it
// into multiply-adds.
struct Sum {
    struct Term {
        int sign;
        std::string coef;  // empty: 1
        std::string var;
    };
    std::vector<Term> t;
    void add(int sg, const std::string& c, const std::string& v) { t.push_back({sg, c, v}); }
    std::string str() const
    {
        if (t.empty()) return "(R)0";
        std::string s;
        for (size_t k = 0; k < t.size(); k++) {
            const std::string prod = t[k].coef.empty() ? t[k].var : t[k].coef + " * " + t[k].var;
            if (k == 0) s += (t[k].sign < 0 ? "-" : "") + prod;
            else s += (t[k].sign < 0 ? " - " : " + ") + prod;
        }
        return s;
    }
};

// (re, im) += e * (vr + i vi)
void cmac(Sum& re, Sum& im, const Coef& e, const std::string& vr, const std::string& vi)
{
    switch (e.cls) {
        case C_ZERO: break;
        case C_ONE: re.add(1, "", vr); im.add(1, "", vi); break;
        case C_MONE: re.add(-1, "", vr); im.add(-1, "", vi); break;
        case C_I: re.add(-1, "", vi); im.add(1, "", vr); break;
        case C_MI: re.add(1, "", vi); im.add(-1, "", vr); break;
        case C_REAL: re.add(1, e.re, vr); im.add(1, e.re, vi); break;
        case C_IMAG: re.add(-1, e.im, vi); im.add(1, e.im, vr); break;
        default:
            re.add(1, e.re, vr);
            re.add(-1, e.im, vi);
            im.add(1, e.re, vi);
            im.add(1, e.im, vr);
            break;
    }
}

std::string hex(uint64_t v)
{
    char b[32];
    std::snprintf(b, sizeof b, "0x%llx", (unsigned long long)v);
    return b;
}

template <typename R>
struct Gen {
    std::ostringstream o;
    const std::vector<R>& par;  // the kernel's parameter block (jit_params)
    int thr_of_tile[16];  // tile bit -> thread index bit of the current phase (-1: register bit)
    int slot[16];         // register index -> variable holding it
    int tmp = 0;
    bool ok = true;
    // Conditional exchanges on a register bit (an X whose controls are thread
    // or CTA bits) not yet applied to the registers: each is folded into the
    // phase's store addresses unless a later op of the phase depends on its bit.
    struct Pend {
        std::string cond;
        int b;
        uint32_t tm = 0;  // thread-index bits the condition requires (0: uniform over the CTA)
    };
    std::vector<Pend> pend;
    int nvec = 1;  // 2 in an adjoint sub-pass: psi in r/q, lambda in u/w, same ops on both
    // Complex64: two register updates with the same coefficients run as one
    // packed FP32x2 instruction each (half the issue slots); pk_order: the
    // register bits to pair amplitudes along, least used by the phase first
    // (when one vector is packed).
    bool pack = false;
    int pk_order[4] = {0, 1, 2, 3};
    // complex64 updates with real coefficients only: real and imaginary parts
    // as one packed pair (decided per phase)
    bool pack_parts = false;
    explicit Gen(const std::vector<R>& p) : par(p) {}
    std::string rv(int m, int v = 0) const { return (v ? "u" : "r") + std::to_string(slot[m]); }
    std::string iv(int m, int v = 0) const { return (v ? "w" : "q") + std::to_string(slot[m]); }
};

// One register update as the generated code writes it: local copies of its
// inputs, then each output variable as a sum over those copies.
struct Blk {
    int i = 0, v = 0;  // register index (the op's loop index) and vector
    std::vector<std::pair<std::string, std::string>> in;  // local name, variable
    std::vector<std::pair<std::string, Sum>> out;         // variable, value
    std::string sig() const
    {
        std::string k;
        for (const auto& x : in) k += x.first + ",";
        for (const auto& x : out) k += x.second.str() + ";";
        return k;
    }
};

// Packed form of a sum: the first plain positive term (else a product) starts
// it, the others follow as packed multiply-adds / adds; kp collects the
// coefficient pairs (the same value in both halves) it needs.
std::string packed_sum(const Sum& s, std::map<std::string, std::string>& kp, int& tmp)
{
    auto K = [&](int sg, const std::string& c) {
        const std::string e = c.empty() ? (sg < 0 ? "-1.0f" : "1.0f") : (sg < 0 ? "-" + c : c);
        auto it = kp.find(e);
        if (it != kp.end()) return it->second;
        const std::string name = "k" + std::to_string(tmp++);
        kp[e] = name;
        return name;
    };
    if (s.t.empty()) return "make_float2(0.0f, 0.0f)";
    std::vector<Sum::Term> t = s.t;
    for (size_t k = 0; k < t.size(); k++)
        if (t[k].coef.empty() && t[k].sign > 0) {
            std::rotate(t.begin(), t.begin() + (long)k, t.begin() + (long)k + 1);
            break;
        }
    std::string acc = (t[0].coef.empty() && t[0].sign > 0) ? t[0].var
                                                            : "__fmul2_rn(" + K(t[0].sign, t[0].coef) + ", " + t[0].var + ")";
    for (size_t k = 1; k < t.size(); k++) {
        if (t[k].coef.empty() && t[k].sign > 0) acc = "__fadd2_rn(" + acc + ", " + t[k].var + ")";
        else acc = "__ffma2_rn(" + K(t[k].sign, t[k].coef) + ", " + t[k].var + ", " + acc + ")";
    }
    return acc;
}

// Does every output pair (real part, imaginary part) of the update compute
// the same sum, the real part over real inputs and the imaginary part over
// the matching imaginary ones (real coefficients only)?
bool parallel_parts(const Blk& b)
{
    if (b.in.size() % 2 || b.out.size() % 2) return false;
    for (size_t k = 0; k < b.in.size(); k += 2) {
        const std::string& a = b.in[k].first;
        const std::string& c = b.in[k + 1].first;
        if (a.empty() || a.back() != 'r' || c != a.substr(0, a.size() - 1) + "i") return false;
    }
    for (size_t k = 0; k < b.out.size(); k += 2) {
        const Sum& re = b.out[k].second;
        const Sum& im = b.out[k + 1].second;
        if (re.t.size() != im.t.size() || re.t.empty()) return false;
        for (size_t j = 0; j < re.t.size(); j++) {
            const auto& x = re.t[j];
            const auto& y = im.t[j];
            if (x.sign != y.sign || x.coef != y.coef || x.var.empty() || x.var.back() != 'r' ||
                y.var != x.var.substr(0, x.var.size() - 1) + "i")
                return false;
        }
    }
    return true;
}

// Print an op's register updates: in pairs of identical updates as packed
// instructions where the generator packs (psi with lambda in an adjoint
// sub-pass, else registers that differ in one bit the op does not touch),
// the rest one by one.
template <typename R>
void flush(Gen<R>& g, std::vector<Blk>& bl)
{
    std::vector<int> mate(bl.size(), -1);
    if (g.pack) {
        std::vector<std::string> sg(bl.size());
        for (size_t a = 0; a < bl.size(); a++) sg[a] = bl[a].sig();
        auto find = [&](int i, int v, const std::string& k) {
            for (size_t c = 0; c < bl.size(); c++)
                if (bl[c].i == i && bl[c].v == v && sg[c] == k) return (int)c;
            return -1;
        };
        if (g.nvec == 2) {
            for (size_t a = 0; a < bl.size(); a++)
                if (bl[a].v == 0 && mate[a] < 0) {
                    const int c = find(bl[a].i, 1, sg[a]);
                    if (c >= 0 && mate[c] < 0) {
                        mate[a] = c;
                        mate[c] = (int)a;
                    }
                }
        } else {
            int best = -1, bestn = 0;
            for (int q = 0; q < 4; q++) {
                const int b = g.pk_order[q];
                int n = 0;
                for (size_t a = 0; a < bl.size(); a++)
                    if (find(bl[a].i ^ (1 << b), bl[a].v, sg[a]) >= 0) n++;
                if (n > bestn) {
                    bestn = n;
                    best = b;
                }
            }
            for (size_t a = 0; best >= 0 && a < bl.size(); a++) {
                if (mate[a] >= 0 || (bl[a].i >> best) & 1) continue;
                const int c = find(bl[a].i ^ (1 << best), bl[a].v, sg[a]);
                if (c >= 0 && mate[c] < 0) {
                    mate[a] = c;
                    mate[c] = (int)a;
                }
            }
        }
    }
    std::map<std::string, std::string> kp;
    std::ostringstream body;
    for (size_t a = 0; a < bl.size(); a++) {
        const Blk& A = bl[a];
        if (mate[a] < 0 && g.pack_parts && parallel_parts(A)) {
            // real coefficients only: the real and imaginary parts of each
            // amplitude see the same sums and run as one packed instruction on
            // the register pair the shared-memory loads fill anyway
            body << "{ const float2 ";
            for (size_t k = 0; k < A.in.size(); k += 2)
                body << (k ? ", " : "") << A.in[k].first.substr(0, A.in[k].first.size() - 1) << " = make_float2("
                     << A.in[k].second << ", " << A.in[k + 1].second << ")";
            body << "; ";
            for (size_t k = 0; k < A.out.size(); k += 2) {
                Sum m = A.out[k].second;
                for (auto& t : m.t) t.var.pop_back();
                body << "const float2 o" << k / 2 << " = " << packed_sum(m, kp, g.tmp) << "; ";
            }
            for (size_t k = 0; k < A.out.size(); k += 2)
                body << A.out[k].first << " = o" << k / 2 << ".x; " << A.out[k + 1].first << " = o" << k / 2 << ".y; ";
            body << "}\n";
            continue;
        }
        if (mate[a] < 0) {
            body << "{ const R ";
            for (size_t k = 0; k < A.in.size(); k++) body << (k ? ", " : "") << A.in[k].first << " = " << A.in[k].second;
            body << "; ";
            for (const auto& x : A.out) body << x.first << " = " << x.second.str() << "; ";
            body << "}\n";
            continue;
        }
        if (mate[a] < (int)a) continue;
        const Blk& B = bl[mate[a]];
        body << "{ const float2 ";
        for (size_t k = 0; k < A.in.size(); k++)
            body << (k ? ", " : "") << A.in[k].first << " = make_float2(" << A.in[k].second << ", " << B.in[k].second
                 << ")";
        body << "; ";
        for (size_t k = 0; k < A.out.size(); k++)
            body << "const float2 o" << k << " = " << packed_sum(A.out[k].second, kp, g.tmp) << "; ";
        for (size_t k = 0; k < A.out.size(); k++)
            body << A.out[k].first << " = o" << k << ".x; " << B.out[k].first << " = o" << k << ".y; ";
        body << "}\n";
    }
    for (const auto& x : kp) g.o << "const float2 " << x.second << " = make_float2(" << x.first << ", " << x.first << ");\n";
    g.o << body.str();
    bl.clear();
}

// Coefficient chosen at run time by `sel` (0..n-1) among candidates whose
// parts sit at params[pidx[k]], params[pidx[k] + 1].
template <typename R>
Coef select_coef(Gen<R>& g, const std::string& sel, const std::vector<size_t>& pidx)
{
    const size_t n = pidx.size();
    bool same = true, real = true, imag = true;
    for (size_t k = 0; k < n; k++) {
        const R re = g.par[pidx[k]], im = g.par[pidx[k] + 1];
        if (re != g.par[pidx[0]] || im != g.par[pidx[0] + 1]) same = false;
        if (im != 0) real = false;
        if (re != 0) imag = false;
    }
    if (same) return fixed_coef<R>(g.par[pidx[0]], g.par[pidx[0] + 1], pidx[0]);
    Coef c;
    c.cls = real ? C_REAL : imag ? C_IMAG : C_GEN;
    auto pick = [&](int part) {
        if (n == 2) return "(" + sel + " ? " + pref(pidx[1] + part) + " : " + pref(pidx[0] + part) + ")";
        return "((" + sel + ") & 2u ? ((" + sel + ") & 1u ? " + pref(pidx[3] + part) + " : " + pref(pidx[2] + part) +
               ") : ((" + sel + ") & 1u ? " + pref(pidx[1] + part) + " : " + pref(pidx[0] + part) + "))";
    };
    const std::string name = "e" + std::to_string(g.tmp++);
    if (c.cls != C_IMAG) {
        g.o << "const R " << name << "r = " << pick(0) << ";\n";
        c.re = name + "r";
    }
    if (c.cls != C_REAL) {
        g.o << "const R " << name << "i = " << pick(1) << ";\n";
        c.im = name + "i";
    }
    return c;
}

// expression of a constant entry-index bit (see kSrcNone); empty for none
template <typename R>
std::string const_bit(Gen<R>& g, uint8_t s)
{
    if (s == kSrcNone) return "";
    if (s < 0x40) {
        const int j = s < 16 ? g.thr_of_tile[s] : -1;
        if (j < 0) {
            g.ok = false;
            return "0u";
        }
        return "((threadIdx.x >> " + std::to_string(j) + ") & 1u)";
    }
    if (s < 0x80) return "(uint32_t)((base >> " + std::to_string(s - 0x40) + ") & 1ull)";
    return "(uint32_t)((gbase >> " + std::to_string(s - 0x80) + ") & 1ull)";
}

// controls that are not register bits: thread bits and bits outside the tile
template <typename R>
std::string op_cond(Gen<R>& g, const PhaseOp<R>& op, const CtaCtrl* ctl)
{
    std::vector<std::string> parts;
    if (op.tmask) {
        uint32_t tm = 0;
        for (int b = 0; b < 16; b++) {
            if (!((op.tmask >> b) & 1u)) continue;
            const int j = g.thr_of_tile[b];
            if (j < 0) g.ok = false;
            else tm |= 1u << j;
        }
        parts.push_back("(threadIdx.x & " + hex(tm) + "u) == " + hex(tm) + "u");
    }
    if (op.flags & 1u) {
        const CtaCtrl cc = ctl[op.aux];
        if (cc.cl) parts.push_back("(base & " + hex(cc.cl) + "ull) == " + hex(cc.cl) + "ull");
        if (cc.cg) parts.push_back("(gbase & " + hex(cc.cg) + "ull) == " + hex(cc.cg) + "ull");
    }
    std::string s;
    for (size_t k = 0; k < parts.size(); k++) s += (k ? " && (" : "(") + parts[k] + ")";
    return s;
}

// thread-index bits an op's controls require (its thread-bit controls)
template <typename R>
uint32_t thread_mask(const Gen<R>& g, const PhaseOp<R>& op)
{
    uint32_t tm = 0;
    for (int b = 0; b < 16; b++)
        if (((op.tmask >> b) & 1u) && g.thr_of_tile[b] >= 0) tm |= 1u << g.thr_of_tile[b];
    return tm;
}

// register bits an op acts on as target or diagonal index
template <typename R>
uint32_t op_bits(const PhaseOp<R>& op)
{
    const uint32_t code = op.code;
    if (code < kCodeDiag2) return 1u << (code & 3);
    if (code < kCodeDiagT) {
        const uint32_t x = (code - kCodeDiag2) & 15;
        return (1u << (x & 3)) | (1u << (x >> 2));
    }
    if (code < kCodeDense2) return 0;
    return (1u << (op.pad & 3)) | (1u << ((op.pad >> 2) & 3));
}

// does the op commute with exchanging the registers that differ in bit x?
template <typename R>
bool symmetric(const PhaseOp<R>& op, int x)
{
    if (op_bits(op) & (1u << x)) return false;
    for (int i = 0; i < 16; i++)
        if (((op.amask >> i) & 1u) != ((op.amask >> (i ^ (1 << x))) & 1u)) return false;
    return true;
}

template <typename R>
void emit_exchange(Gen<R>& g, const std::string& cond, int b)
{
    g.o << "if (" << cond << ") {\n";
    for (int v = 0; v < g.nvec; v++)
        for (int i = 0; i < 16; i++) {
            if (i & (1 << b)) continue;
            const int j = i | (1 << b);
            g.o << "{ const R tr = " << g.rv(i, v) << ", ti = " << g.iv(i, v) << "; " << g.rv(i, v) << " = "
                << g.rv(j, v) << "; " << g.iv(i, v) << " = " << g.iv(j, v) << "; " << g.rv(j, v) << " = tr; "
                << g.iv(j, v) << " = ti; }\n";
        }
    g.o << "}\n";
}

// Before an op: a pending exchange on bit b stays pending if the op commutes
// with it, or if the op acts on b as its target or diagonal index (a 2x2 or
// diagonal op whose controls do not involve b): the op is then applied
// conjugated by the exchange, X U X, whose entries are U's with the b index
// flipped, chosen per thread (returned); otherwise it is applied now.
template <typename R>
std::vector<typename Gen<R>::Pend> settle(Gen<R>& g, const PhaseOp<R>& op)
{
    std::vector<typename Gen<R>::Pend> keep, conj;
    const bool conjugable = op.code < kCodeDiagT;  // 2x2, one- or two-register diagonal
    for (const auto& pd : g.pend) {
        if (symmetric(op, pd.b)) {
            keep.push_back(pd);
        } else if (conjugable && ((op_bits(op) >> pd.b) & 1u)) {
            keep.push_back(pd);
            conj.push_back(pd);
        } else {
            emit_exchange(g, pd.cond, pd.b);
        }
    }
    g.pend.swap(keep);
    return conj;
}

// selector expression over pending exchanges: bit j set when conj[j] holds
template <typename R>
std::string flip_sel(const std::vector<typename Gen<R>::Pend>& conj)
{
    std::string s;
    for (size_t j = 0; j < conj.size(); j++)
        s += (j ? " | " : "") + std::string("((") + conj[j].cond + ") ? " + std::to_string(1u << j) + "u : 0u)";
    return "(" + s + ")";
}

// register m *= e
template <typename R>
void mul_reg(Gen<R>& g, std::vector<Blk>& bl, int m, const Coef& e)
{
    if (e.cls == C_ONE) return;
    Sum re, im;
    cmac(re, im, e, "xr", "xi");
    for (int v = 0; v < g.nvec; v++) {
        Blk b;
        b.i = m;
        b.v = v;
        b.in = {{"xr", g.rv(m, v)}, {"xi", g.iv(m, v)}};
        b.out = {{g.rv(m, v), re}, {g.iv(m, v), im}};
        bl.push_back(std::move(b));
    }
}

template <typename R>
void emit_dense1(Gen<R>& g, const PhaseOp<R>& op, size_t pb, int b, const std::string& cond,
                 const std::vector<typename Gen<R>::Pend>& conj)
{
    const R* m = g.par.data() + pb;  // the op's entries as the kernel reads them
    const bool ident = m[0] == 1 && m[1] == 0 && m[2] == 0 && m[3] == 0 && m[4] == 0 && m[5] == 0 && m[6] == 1 &&
                       m[7] == 0;
    if (ident) return;
    const bool xperm = m[0] == 0 && m[1] == 0 && m[2] == 1 && m[3] == 0 && m[4] == 1 && m[5] == 0 && m[6] == 0 &&
                       m[7] == 0;
    if (xperm && cond.empty()) {
        for (int i = 0; i < 16; i++)
            if ((op.amask >> i) & 1u) std::swap(g.slot[i], g.slot[i | (1 << b)]);
        return;
    }
    uint32_t leaders = 0;  // every pair of bit b: an exchange of all of them can wait for the stores
    for (int i = 0; i < 16; i++)
        if (!(i & (1 << b))) leaders |= 1u << i;
    if (xperm && op.amask == leaders) {
        // at most three pending, on distinct bits (their store bases are the
        // eight sign combinations); apply the oldest otherwise
        for (size_t k = 0; k < g.pend.size();) {
            if (g.pend[k].b == b || g.pend.size() >= 3) {
                emit_exchange(g, g.pend[k].cond, g.pend[k].b);
                g.pend.erase(g.pend.begin() + (long)k);
            } else {
                k++;
            }
        }
        g.pend.push_back({cond, b, thread_mask(g, op)});
        return;
    }
    Coef e[4];
    if (conj.empty()) {
        for (int k = 0; k < 4; k++) e[k] = fixed_coef<R>(m[2 * k], m[2 * k + 1], pb + 2 * k);
    } else {
        // X U X: row and column index flipped (entry k -> k ^ 3)
        const std::string sel = flip_sel<R>(conj);
        for (int k = 0; k < 4; k++) e[k] = select_coef(g, sel, {pb + 2 * (size_t)k, pb + 2 * (size_t)(k ^ 3)});
    }
    if (!cond.empty()) g.o << "if (" << cond << ") {\n";
    std::vector<Blk> bl;
    for (int i = 0; i < 16; i++) {
        if (!((op.amask >> i) & 1u)) continue;
        const int j = i | (1 << b);
        Sum xr, xi, yr, yi;
        cmac(xr, xi, e[0], "xr", "xi");
        cmac(xr, xi, e[1], "yr", "yi");
        cmac(yr, yi, e[2], "xr", "xi");
        cmac(yr, yi, e[3], "yr", "yi");
        for (int v = 0; v < g.nvec; v++) {
            Blk k;
            k.i = i;
            k.v = v;
            k.in = {{"xr", g.rv(i, v)}, {"xi", g.iv(i, v)}, {"yr", g.rv(j, v)}, {"yi", g.iv(j, v)}};
            k.out = {{g.rv(i, v), xr}, {g.iv(i, v), xi}, {g.rv(j, v), yr}, {g.iv(j, v), yi}};
            bl.push_back(std::move(k));
        }
    }
    flush(g, bl);
    if (!cond.empty()) g.o << "}\n";
}

template <typename R>
void emit_diag2(Gen<R>& g, const PhaseOp<R>& op, size_t pb, int b0, int b1, const std::string& cond,
                const std::vector<typename Gen<R>::Pend>& conj)
{
    Coef e[4];
    bool all_one = true;
    for (int v = 0; v < 4; v++)
        if (entry_class(g.par[pb + 2 * v], g.par[pb + 2 * v + 1]) != C_ONE) all_one = false;
    if (all_one) return;
    const std::string sel = conj.empty() ? std::string() : flip_sel<R>(conj);
    for (int v = 0; v < 4; v++) {
        if (conj.empty()) {
            e[v] = fixed_coef<R>(g.par[pb + 2 * v], g.par[pb + 2 * v + 1], pb + 2 * v);
            continue;
        }
        // a pending exchange on b0 (b1) flips entry-index bit 0 (1)
        std::vector<size_t> cand;
        for (uint32_t c = 0; c < (1u << conj.size()); c++) {
            int w = v;
            for (size_t j = 0; j < conj.size(); j++)
                if ((c >> j) & 1u) w ^= conj[j].b == b0 ? 1 : 2;
            cand.push_back(pb + 2 * (size_t)w);
        }
        e[v] = select_coef(g, sel, cand);
    }
    if (!cond.empty()) g.o << "if (" << cond << ") {\n";
    std::vector<Blk> bl;
    for (int i = 0; i < 16; i++) {
        if (!((op.amask >> i) & 1u)) continue;
        mul_reg(g, bl, i, e[((i >> b0) & 1) | (((i >> b1) & 1) << 1)]);
    }
    flush(g, bl);
    if (!cond.empty()) g.o << "}\n";
}

template <typename R>
void emit_diag1(Gen<R>& g, const PhaseOp<R>& op, size_t pb, int b0, const std::string& cond,
                const std::vector<typename Gen<R>::Pend>& conj)
{
    const std::string cb = const_bit(g, op.csrc);
    auto entry = [&](int rb, int c) { return op.rsel ? (c | (rb << 1)) : (rb | (c << 1)); };
    if (!cond.empty()) g.o << "if (" << cond << ") {\n";
    Coef e[2];
    const std::string fs = conj.empty() ? std::string() : "(" + conj[0].cond + ")";  // flips the register bit
    for (int rb = 0; rb < 2; rb++) {
        if (cb.empty() && fs.empty()) {
            const int v = entry(rb, 0);
            e[rb] = fixed_coef<R>(g.par[pb + 2 * v], g.par[pb + 2 * v + 1], pb + 2 * v);
        } else if (fs.empty()) {
            e[rb] = select_coef(g, cb, {pb + 2 * (size_t)entry(rb, 0), pb + 2 * (size_t)entry(rb, 1)});
        } else if (cb.empty()) {
            e[rb] = select_coef(g, fs, {pb + 2 * (size_t)entry(rb, 0), pb + 2 * (size_t)entry(rb ^ 1, 0)});
        } else {
            e[rb] = select_coef(g, "(" + cb + " | (" + fs + " ? 2u : 0u))",
                                {pb + 2 * (size_t)entry(rb, 0), pb + 2 * (size_t)entry(rb, 1),
                                 pb + 2 * (size_t)entry(rb ^ 1, 0), pb + 2 * (size_t)entry(rb ^ 1, 1)});
        }
    }
    std::vector<Blk> bl;
    for (int i = 0; i < 16; i++) {
        if (!((op.amask >> i) & 1u)) continue;
        mul_reg(g, bl, i, e[(i >> b0) & 1]);
    }
    flush(g, bl);
    if (!cond.empty()) g.o << "}\n";
}

template <typename R>
void emit_diagt(Gen<R>& g, const PhaseOp<R>& op, size_t pb, const std::string& cond)
{
    const std::string c0 = const_bit(g, op.csrc), c1 = const_bit(g, op.csrc1);
    if (!cond.empty()) g.o << "if (" << cond << ") {\n";
    Coef e;
    if (c0.empty() && c1.empty()) e = fixed_coef<R>(g.par[pb], g.par[pb + 1], pb);
    else if (c1.empty()) e = select_coef(g, c0, {pb, pb + 2});
    else if (c0.empty()) e = select_coef(g, c1, {pb, pb + 4});
    else e = select_coef(g, "(" + c0 + " | (" + c1 + " << 1))", {pb, pb + 2, pb + 4, pb + 6});
    std::vector<Blk> bl;
    for (int i = 0; i < 16; i++)
        if ((op.amask >> i) & 1u) mul_reg(g, bl, i, e);
    flush(g, bl);
    if (!cond.empty()) g.o << "}\n";
}

template <typename R>
void emit_dense2(Gen<R>& g, const PhaseOp<R>& op, size_t pb, const std::string& cond)
{
    const int b0 = op.pad & 3, b1 = (op.pad >> 2) & 3;
    Coef e[16];
    for (int k = 0; k < 16; k++) e[k] = fixed_coef<R>(g.par[pb + 2 * k], g.par[pb + 2 * k + 1], pb + 2 * k);
    if (!cond.empty()) g.o << "if (" << cond << ") {\n";
    std::vector<Blk> bl;
    for (int i = 0; i < 16; i++) {
        if (!((op.amask >> i) & 1u)) continue;
        int idx[4];
        for (int k = 0; k < 4; k++) idx[k] = i | ((k & 1) << b0) | (((k >> 1) & 1) << b1);
        for (int vv = 0; vv < g.nvec; vv++) {
            Blk bk;
            bk.i = i;
            bk.v = vv;
            for (int k = 0; k < 4; k++) {
                bk.in.push_back({"v" + std::to_string(k) + "r", g.rv(idx[k], vv)});
                bk.in.push_back({"v" + std::to_string(k) + "i", g.iv(idx[k], vv)});
            }
            for (int r = 0; r < 4; r++) {
                Sum re, im;
                for (int k = 0; k < 4; k++)
                    cmac(re, im, e[4 * r + k], "v" + std::to_string(k) + "r", "v" + std::to_string(k) + "i");
                bk.out.push_back({g.rv(idx[r], vv), re});
                bk.out.push_back({g.iv(idx[r], vv), im});
            }
            bl.push_back(std::move(bk));
        }
    }
    flush(g, bl);
    if (!cond.empty()) g.o << "}\n";
}

// Adjoint: this thread's part of Im<lambda| G |psi> for the generator G (1 X,
// 2 Y, 3 Z) on register bit b, taken before the op is applied: summed over
// the thread's pairs and over the warp by shuffles in R, added to the warp's
// own entry of the slot (shared memory, in R, over the CTA's tiles); the
// kernel sums a slot's warp entries in FP64 at its end (GB300's FP64 pipe is
// narrow: nothing FP64 runs per tile). A pending exchange on b (registers hold X psi, X lambda on
// the threads where it holds) flips the sign for Y and Z (X Y X = -Y, X Z X = -Z).
template <typename R>
void emit_grad(Gen<R>& g, int b, int gen, int slot, const std::vector<typename Gen<R>::Pend>& conj)
{
    g.o << "{ R gp = (R)0;\n";
    for (int i = 0; i < 16; i++) {
        if (i & (1 << b)) continue;
        const int j = i | (1 << b);
        const std::string p0r = g.rv(i, 0), p0i = g.iv(i, 0), p1r = g.rv(j, 0), p1i = g.iv(j, 0);
        const std::string l0r = g.rv(i, 1), l0i = g.iv(i, 1), l1r = g.rv(j, 1), l1i = g.iv(j, 1);
        if (gen == 1)  // conj(l0) p1 + conj(l1) p0
            g.o << "gp += " << l0r << " * " << p1i << " - " << l0i << " * " << p1r << " + " << l1r << " * " << p0i
                << " - " << l1i << " * " << p0r << ";\n";
        else if (gen == 2)  // conj(l0)(-i p1) + conj(l1)(i p0): Im = -Re(conj(l0) p1) + Re(conj(l1) p0)
            g.o << "gp += " << l1r << " * " << p0r << " + " << l1i << " * " << p0i << " - " << l0r << " * " << p1r
                << " - " << l0i << " * " << p1i << ";\n";
        else  // conj(l0) p0 - conj(l1) p1
            g.o << "gp += " << l0r << " * " << p0i << " - " << l0i << " * " << p0r << " - " << l1r << " * " << p1i
                << " + " << l1i << " * " << p1r << ";\n";
    }
    for (const auto& pd : conj)
        if (pd.b == b && gen != 1) g.o << "if (" << pd.cond << ") gp = -gp;\n";
    g.o << "gp += __shfl_xor_sync(0xffffffffu, gp, 16); gp += __shfl_xor_sync(0xffffffffu, gp, 8); "
           "gp += __shfl_xor_sync(0xffffffffu, gp, 4); gp += __shfl_xor_sync(0xffffffffu, gp, 2); "
           "gp += __shfl_xor_sync(0xffffffffu, gp, 1);\n"
        << "if ((threadIdx.x & 31u) == 0u) gw[" << slot << " * 8 + (threadIdx.x >> 5)] += gp; }\n";
}

template <typename R> struct RName;
template <> struct RName<float> {
    static constexpr const char* r = "float";
    static constexpr const char* t = "float2";
    static constexpr int minb = 3, minb_adj = 2;
};
template <> struct RName<double> {
    static constexpr const char* r = "double";
    static constexpr const char* t = "double2";
    static constexpr int minb = 2, minb_adj = 1;
};

// ------------------------------------------------------------ NVRTC / driver
struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t*) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char*) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram*) = nullptr;
};

Nvrtc load_nvrtc()
{
    Nvrtc n;
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    if (const char* h = std::getenv("CUDA_HOME")) names.push_back(std::string(h) + "/lib64/libnvrtc.so.13");
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void* lib = nullptr;
    for (const std::string& nm : names)
        if ((lib = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) {
        n.why = "libnvrtc.so.13 not found";
        return n;
    }
    bool ok = true;
    auto sym = [&](const char* s) {
        void* p = dlsym(lib, s);
        if (!p) ok = false;
        return p;
    };
    n.create = reinterpret_cast<decltype(n.create)>(sym("nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(sym("nvrtcCompileProgram"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(sym("nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(sym("nvrtcGetCUBIN"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(sym("nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(sym("nvrtcGetProgramLog"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(sym("nvrtcDestroyProgram"));
    n.ok = ok;
    if (!ok) n.why = "libnvrtc lacks an expected entry point";
    return n;
}

Nvrtc& nvrtc()
{
    static Nvrtc n = load_nvrtc();
    return n;
}

struct Drv {
    bool ok = false;
    std::string why;
    CUresult (*load)(CUmodule*, const void*) = nullptr;
    CUresult (*getfn)(CUfunction*, CUmodule, const char*) = nullptr;
    CUresult (*setattr)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                       void**, void**) = nullptr;
};

Drv load_drv()
{
    Drv d;
    bool ok = true;
    auto sym = [&](const char* s) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion(s, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            ok = false;
        return p;
    };
    d.load = reinterpret_cast<decltype(d.load)>(sym("cuModuleLoadData"));
    d.getfn = reinterpret_cast<decltype(d.getfn)>(sym("cuModuleGetFunction"));
    d.setattr = reinterpret_cast<decltype(d.setattr)>(sym("cuFuncSetAttribute"));
    d.launch = reinterpret_cast<decltype(d.launch)>(sym("cuLaunchKernel"));
    d.ok = ok;
    if (!ok) d.why = "CUDA driver entry points unavailable";
    return d;
}

Drv& drv()
{
    static Drv d = load_drv();
    return d;
}

std::mutex g_mu;
std::unordered_map<std::string, std::unique_ptr<JitFn>> g_cache;  // key: device, arch, source

struct Job {
    size_t index = 0;
    const std::string* src = nullptr;
    std::string key;
    std::string cubin;
    std::string log;
    bool ok = false;
};

void compile_one(Job& j, const std::string& arch_opt)
{
    Nvrtc& n = nvrtc();
    nvrtcProgram prog;
    if (n.create(&prog, j.src->c_str(), "sv_subpass.cu", kJitHeaderCount, kJitHeaders, kJitHeaderNames) !=
        NVRTC_SUCCESS) {
        j.log = "nvrtcCreateProgram failed";
        return;
    }
    const char* opts[] = {arch_opt.c_str(), "--std=c++17"};
    const nvrtcResult r = n.compile(prog, 2, opts);
    size_t ls = 0;
    n.log_size(prog, &ls);
    if (ls > 1) {
        j.log.resize(ls);
        n.log(prog, &j.log[0]);
    }
    if (r == NVRTC_SUCCESS) {
        size_t cs = 0;
        n.cubin_size(prog, &cs);
        j.cubin.resize(cs);
        if (cs && n.cubin(prog, &j.cubin[0]) == NVRTC_SUCCESS) j.ok = true;
    }
    n.destroy(&prog);
}

}  // namespace

// An op applied to every amplitude of the tile: no controls outside its
// registers' pair structure and none among them.
template <typename R>
bool uncontrolled(const PhaseOp<R>& op)
{
    if (op.flags || op.tmask) return false;
    uint32_t all = 0xffffu;
    if (op.code < kCodeDiag2 && op.code / 8 != PK_DIAG1) {
        all = 0;  // 2x2: the pair leaders of the target bit
        for (int i = 0; i < 16; i++)
            if (!(i & (1 << (op.code & 3)))) all |= 1u << i;
    } else if (op.code == kCodeDense2) {
        all = 0;
        const int b0 = op.pad & 3, b1 = (op.pad >> 2) & 3;
        for (int i = 0; i < 16; i++)
            if (!(i & ((1 << b0) | (1 << b1)))) all |= 1u << i;
    }
    return op.amask == all;
}

template <typename R>
void jit_params(const Phase* ph, int nph, const PhaseOp<R>* ops, const R* d2m, std::vector<R>& params, bool factor)
{
    using C = std::complex<double>;
    params.clear();
    // each op's entries in order; an uncontrolled op U is stored as U / a,
    // with a its first entry (so that the entry becomes exactly 1 and the
    // generated code skips its multiplies) unless that entry is under a
    // quarter of the largest, then the largest; the product of those factors
    // is multiplied into the last such op instead. The choice of entry changes
    // only for rotations near pi. With |a| >= |largest| / 4, U / a scales
    // amplitudes by at most 4 x (entries per row): 2^3 for a 2x2, 2^2 for a
    // diagonal, 2^4 for a 4x4; ops are factored while the sum of those bounds
    // stays within 2^120 (inside the FP32 range; a bound on the structure, so
    // small changes of the angles do not change which ops are factored).
    struct Norm {
        size_t at;
        int n;
        C a;
    };
    std::vector<Norm> norm;
    int growth = 0;  // log2 of the bound on the amplitudes' growth so far
    for (int pi = 0; pi < nph; pi++)
        for (int oi = ph[pi].op_begin; oi < ph[pi].op_begin + ph[pi].op_count; oi++) {
            const PhaseOp<R>& op = ops[oi];
            const size_t at = params.size();
            const int n = op.code == kCodeDense2 ? 16 : 4;
            if (op.code == kCodeDense2) params.insert(params.end(), d2m + 32ull * op.aux, d2m + 32ull * op.aux + 32);
            else params.insert(params.end(), op.m, op.m + 8);
            if (!factor || !uncontrolled(op)) continue;
            C big(0, 0);
            for (int k = 0; k < n; k++) {
                const C e((double)params[at + 2 * k], (double)params[at + 2 * k + 1]);
                if (std::abs(e) > std::abs(big)) big = e;
            }
            const C first((double)params[at], (double)params[at + 1]);
            const C a = std::abs(first) >= 0.25 * std::abs(big) ? first : big;
            if (std::abs(a) == 0 || a == C(1, 0)) continue;
            const int g = n == 16 ? 4 : (op.code < kCodeDiag2 && op.code / 8 != PK_DIAG1) ? 3 : 2;
            if (growth + g > 120) continue;
            growth += g;
            norm.push_back({at, n, a});
        }
    if (!norm.empty()) {
        C rest(1, 0);
        for (size_t j = 0; j + 1 < norm.size(); j++) rest *= norm[j].a;
        for (size_t j = 0; j < norm.size(); j++) {
            const C f = j + 1 < norm.size() ? C(1, 0) / norm[j].a : rest;
            for (int k = 0; k < norm[j].n; k++) {
                R* e = &params[norm[j].at + 2 * k];
                const C x((double)e[0], (double)e[1]);
                // an entry equal to the factor becomes exactly 1 (complex
                // division would leave a rounding residue in its imaginary part)
                const C v = (j + 1 < norm.size() && x == norm[j].a) ? C(1, 0) : x * f;
                e[0] = (R)v.real();
                e[1] = (R)v.imag();
            }
        }
    }
    if (params.empty()) params.push_back((R)0);
}

// The last phase of a sub-pass that does not encode stores its registers
// straight to HBM (no shared-memory round trip) when its thread bits 0 and 1
// are tile bits 0 and 1: four consecutive lanes then write one whole 32-byte
// sector (complex64). An adjoint sub-pass stores psi and lambda so.
bool direct_store(const Phase* ph, int nph, bool enc)
{
    return !enc && nph > 0 && ph[nph - 1].tpos[0] == 0 && ph[nph - 1].tpos[1] == 1;
}

// Which pending exchanges to fold into a phase's store addresses (1) rather
// than apply in registers (0): the choice with the least cost, counting an
// exchange in registers as 64 issue cycles of a 256-thread tile (32 selects
// per thread) and each extra shared-memory wavefront of the stores (bank
// pairs shared within a half-warp, padded layout: slot mod 16) as one.
template <typename R>
std::vector<int> fold_plan(const Gen<R>& g, const Phase& P, const uint32_t* K)
{
    const size_t np = g.pend.size();
    std::vector<int> best(np, 1);
    bool lanes = false;  // any condition on lane bits 0..3?
    for (const auto& pd : g.pend)
        if (pd.tm & 15u) lanes = true;
    if (!lanes) return best;
    long best_cost = -1;
    for (uint32_t f = 0; f < (1u << np); f++) {
        long cost = 0;
        for (size_t j = 0; j < np; j++)
            if (!((f >> j) & 1)) cost += 64;
        // extra wavefronts of the 16 stores over the CTA's 16 half-warps
        for (int m = 0; m < 16; m++)
            for (int hw = 0; hw < 16; hw++) {
                int count[16] = {};
                uint32_t seen[16][16];
                int worst = 1;
                for (int l = 0; l < 16; l++) {
                    const uint32_t t = 16u * hw + l;
                    uint32_t tb = 0;
                    for (int j = 0; j < kPhaseTileQubits - kPhaseRegBits; j++)
                        if ((t >> j) & 1u) tb |= 1u << P.tpos[j];
                    int64_t slot = (int64_t)pad_slot(tb) + K[m];
                    for (size_t j = 0; j < np; j++) {
                        if (!((f >> j) & 1) || (t & g.pend[j].tm) != g.pend[j].tm) continue;
                        const int64_t dlt = pad_slot(1u << P.rpos[g.pend[j].b]);
                        slot += ((m >> g.pend[j].b) & 1) ? -dlt : dlt;
                    }
                    const uint32_t bank = (uint32_t)(slot & 15), sl = (uint32_t)slot;
                    bool dup = false;
                    for (int q = 0; q < count[bank]; q++)
                        if (seen[bank][q] == sl) dup = true;
                    if (!dup) {
                        seen[bank][count[bank]++] = sl;
                        worst = std::max(worst, count[bank]);
                    }
                }
                cost += worst - 1;
            }
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            for (size_t j = 0; j < np; j++) best[j] = (f >> j) & 1;
        }
    }
    return best;
}

template <typename R>
void jit_key(const Phase* ph, int nph, const PhaseOp<R>* ops, const CtaCtrl* ctl, const std::vector<R>& params,
             bool dec, bool enc, const TileDesc& td, std::string& key, const int32_t* grad)
{
    size_t pb = 0;
    key.clear();
    auto put = [&](const void* p, size_t n) { key.append(static_cast<const char*>(p), n); };
    const uint8_t hdr[kKeyHeader] = {(uint8_t)sizeof(R), (uint8_t)dec, (uint8_t)enc, (uint8_t)(grad ? 2 : 1),
                                     (uint8_t)td.l};
    put(hdr, kKeyHeader);
    // the direct stores' and the tile prefetch's offsets are compiled in
    if (direct_store(ph, nph, enc) || (!grad && prefetches(dec, sizeof(R)))) put(td.hpos, (size_t)(td.t - td.l));
    for (int pi = 0; pi < nph; pi++) {
        const Phase& P = ph[pi];
        put(P.tpos, sizeof P.tpos);
        put(P.sroff, sizeof P.sroff);
        put(&P.op_count, sizeof P.op_count);
        for (int oi = P.op_begin; oi < P.op_begin + P.op_count; oi++) {
            const PhaseOp<R>& op = ops[oi];
            put(&op.code, 2);
            put(&op.amask, 2);
            put(&op.tmask, 2);
            put(&op.flags, 1);
            put(&op.csrc, 1);
            put(&op.csrc1, 1);
            put(&op.rsel, 1);
            put(&op.pad, 2);
            if (grad) put(&grad[oi], sizeof(int32_t));
            if (op.flags & 1u) put(&ctl[op.aux], sizeof(CtaCtrl));
            // the value-dependent choices of the generator: each entry's class
            // and, for 2x2 / diagonal ops, which entries are equal
            const bool d2 = op.code == kCodeDense2;
            const R* v = params.data() + pb;
            pb += d2 ? 32 : 8;
            const int ne = d2 ? 16 : 4;
            for (int k = 0; k < ne; k++) key.push_back((char)entry_class(v[2 * k], v[2 * k + 1]));
            if (!d2) {
                uint8_t eq = 0;
                int bit = 0;
                for (int a = 0; a < 4; a++)
                    for (int b = a + 1; b < 4; b++, bit++)
                        if (v[2 * a] == v[2 * b] && v[2 * a + 1] == v[2 * b + 1]) eq |= (uint8_t)(1u << bit);
                key.push_back((char)eq);
            }
        }
    }
}

template <typename R>
std::string jit_source(const Phase* ph, int nph, const PhaseOp<R>* ops, const CtaCtrl* ctl, const R* d2m, bool dec,
                       bool enc, const TileDesc& td, const std::vector<R>& params, const int32_t* grad)
{
    const int lrow = td.l;
    (void)d2m;
    Gen<R> g(params);
    const bool adj = grad != nullptr;
    const bool ds = direct_store(ph, nph, enc);
    g.nvec = adj ? 2 : 1;
    int nslot = 0;
    std::ostringstream body, hoist;
    size_t pb = 0;  // parameter slot of the current op (8 values, 32 for a 4x4)
    for (int pi = 0; pi < nph; pi++) {
        const Phase& P = ph[pi];
        for (int b = 0; b < 16; b++) g.thr_of_tile[b] = -1;
        std::string tb;
        for (int j = 0; j < kPhaseTileQubits - kPhaseRegBits; j++) {
            g.thr_of_tile[P.tpos[j]] = j;
            tb += (j ? " | " : "") + std::string("(((threadIdx.x >> ") + std::to_string(j) + ") & 1u) << " +
                  std::to_string(P.tpos[j]) + ")";
        }
        for (int m = 0; m < 16; m++) g.slot[m] = m;
        // packing pays in adjoint sub-passes (psi and lambda updates pair up
        // as they are); pairing registers of one vector costs as many register
        // moves and split shared loads as it saves multiply-adds
        g.pack = sizeof(R) == 4 && adj;
        {
            // pair registers along the bits the phase's ops touch least
            int use[4] = {0, 0, 0, 0};
            for (int oi = P.op_begin; oi < P.op_begin + P.op_count; oi++)
                for (int b = 0; b < 4; b++)
                    if (!symmetric(ops[oi], b)) use[b]++;
            for (int q = 0; q < 4; q++) g.pk_order[q] = q;
            std::stable_sort(g.pk_order, g.pk_order + 4, [&](int a, int b) { return use[a] < use[b]; });
        }
        {
            // pairing real and imaginary parts pays where real 2x2 gates (H,
            // RY) outnumber complex diagonals in the phase; measured: -4 % on
            // random layers, +8 % on QFT (mostly controlled phases) when
            // always on
            int nreal = 0, ndiag = 0;
            for (int oi = P.op_begin; oi < P.op_begin + P.op_count; oi++) {
                const uint32_t code = ops[oi].code;
                if (code < kCodeDiag2 && code / 8 == PK_REAL) nreal++;
                else if (code < kCodeDense2 && !(code < kCodeDiag2 && code / 8 != PK_DIAG1)) ndiag++;
            }
            g.pack_parts = sizeof(R) == 4 && nreal > 0 && nreal >= ndiag;
        }
        // padded slot of register index m relative to the thread's base
        uint32_t K[16];
        for (int m = 0; m < 16; m++) {
            uint32_t o = 0;
            for (int q = 0; q < kPhaseRegBits; q++)
                if ((m >> q) & 1) o |= 1u << P.rpos[q];
            K[m] = pad_slot(o);
        }
        g.o.str("");
        // the thread's slot base of this phase does not depend on the tile:
        // computed once per kernel (hoisted), offset by the buffer per tile
        hoist << "const uint32_t tb" << pi << " = " << tb << ";\nconst uint32_t sbb" << pi << " = tb" << pi
              << " + (tb" << pi << " >> 4) + (tb" << pi << " >> 8);\n";
        g.o << "{\nconst uint32_t sb = sbb" << pi << " + bo;\n";
        for (int v = 0; v < g.nvec; v++) {
            g.o << "R ";
            for (int m = 0; m < 16; m++) g.o << (m ? ", " : "") << g.rv(m, v) << ", " << g.iv(m, v);
            g.o << ";\n";
            for (int m = 0; m < 16; m++)
                g.o << "{ const T v = " << (v ? "sl" : "s") << "[sb + " << K[m] << "u]; " << g.rv(m, v)
                    << " = v.x; " << g.iv(m, v) << " = v.y; }\n";
        }
        for (int oi = P.op_begin; oi < P.op_begin + P.op_count; oi++) {
            const PhaseOp<R>& op = ops[oi];
            const std::string cond = op_cond(g, op, ctl);
            const uint32_t code = op.code;
            const auto conj = settle(g, op);
            if (adj && grad[oi] >= 0) {
                // a parameterised RX / RY (2x2) or RZ (one-register diagonal) on register bit code & 3
                if (code >= kCodeDiag2) g.ok = false;
                emit_grad(g, (int)(code & 3), grad[oi] & 3, grad[oi] >> 2, conj);
                nslot = std::max(nslot, (grad[oi] >> 2) + 1);
            }
            if (code < kCodeDiag2) {
                const uint32_t kind = code / 8, b0 = code & 3;
                if (kind == PK_DIAG1) emit_diag1(g, op, pb, (int)b0, cond, conj);
                else emit_dense1(g, op, pb, (int)b0, cond, conj);
            } else if (code < kCodeDiagT) {
                const uint32_t x = (code - kCodeDiag2) & 15;
                emit_diag2(g, op, pb, (int)(x & 3), (int)(x >> 2), cond, conj);
            } else if (code < kCodeDense2) {
                emit_diagt(g, op, pb, cond);
            } else if (code == kCodeDense2) {
                emit_dense2(g, op, pb, cond);
            } else {
                g.ok = false;
            }
            pb += code == kCodeDense2 ? 32 : 8;
        }
        if (!(ds && pi + 1 == nph) && !g.pend.empty()) {
            // a folded exchange conditional on lane bits shifts some lanes'
            // store slots: where that makes two lanes of a half-warp share a
            // bank pair, exchanging in registers (selects) is cheaper than the
            // extra shared-memory wavefronts
            const std::vector<int> how = fold_plan(g, P, K);
            std::vector<typename Gen<R>::Pend> keep;
            for (size_t j = 0; j < g.pend.size(); j++)
                if (how[j]) keep.push_back(g.pend[j]);
                else emit_exchange(g, g.pend[j].cond, g.pend[j].b);
            g.pend.swap(keep);
        }
        const size_t np = g.pend.size();
        if (ds && pi + 1 == nph) {
            // straight to HBM: tile bit b is local bit b below the rows' width,
            // hpos[b - l] above; offsets are additive over disjoint bits like
            // the padded layout, so a pending exchange moves the thread's base
            auto sh = [&](int b) { return b < lrow ? b : (int)td.hpos[b - lrow]; };
            std::string gt;
            for (int j = 0; j < kPhaseTileQubits - kPhaseRegBits; j++)
                gt += (j ? " | " : "") + std::string("((uint64_t)((threadIdx.x >> ") + std::to_string(j) +
                      ") & 1u) << " + std::to_string(sh(P.tpos[j])) + ")";
            hoist << "const uint64_t gth = " << gt << ";\n";
            for (size_t j = 0; j < np; j++)
                g.o << "const int64_t e" << j << " = (" << g.pend[j].cond << ") ? (int64_t)" << hex(1ull << sh(P.rpos[g.pend[j].b]))
                    << "ll : 0ll;\n";
            for (int v = 0; v < g.nvec; v++) {
                const std::string gp = v ? "gl" : "gq";
                g.o << "T* const " << gp << " = " << (v ? "lam" : "amps") << " + base + gth;\n";
                for (uint32_t c = 0; np && c < (1u << np); c++) {
                    g.o << "T* const " << gp << c << " = " << gp;
                    for (size_t j = 0; j < np; j++) g.o << (((c >> j) & 1) ? " - e" : " + e") << j;
                    g.o << ";\n";
                }
                for (int m = 0; m < 16; m++) {
                    uint64_t off = 0;
                    uint32_t c = 0;
                    for (int q = 0; q < kPhaseRegBits; q++)
                        if ((m >> q) & 1) off |= 1ull << sh(P.rpos[q]);
                    for (size_t j = 0; j < np; j++) c |= (uint32_t)((m >> g.pend[j].b) & 1) << j;
                    g.o << (np ? gp + std::to_string(c) : gp) << "[" << hex(off) << "ull] = tile::mk2<T, R>("
                        << g.rv(m, v) << ", " << g.iv(m, v) << ");\n";
                }
            }
            g.pend.clear();
            g.o << "}\n";
            body << g.o.str();
            continue;
        }
        // a pending exchange on register bit b sends register m to the slot of
        // m ^ (1 << b), i.e. K[m] +- pad_slot(1 << rpos[b]) (the layout is
        // additive over disjoint bits): one base per sign combination
        for (size_t j = 0; j < np; j++)
            g.o << "const uint32_t d" << j << " = (" << g.pend[j].cond << ") ? "
                << pad_slot(1u << P.rpos[g.pend[j].b]) << "u : 0u;\n";
        for (uint32_t c = 0; np && c < (1u << np); c++) {
            g.o << "const uint32_t sb" << c << " = sb";
            for (size_t j = 0; j < np; j++) g.o << (((c >> j) & 1) ? " - d" : " + d") << j;
            g.o << ";\n";
        }
        for (int v = 0; v < g.nvec; v++)
            for (int m = 0; m < 16; m++) {
                uint32_t c = 0;
                for (size_t j = 0; j < np; j++) c |= (uint32_t)((m >> g.pend[j].b) & 1) << j;
                g.o << (v ? "sl[" : "s[") << (np ? "sb" + std::to_string(c) : std::string("sb")) << " + " << K[m]
                    << "u] = tile::mk2<T, R>(" << g.rv(m, v) << ", " << g.iv(m, v) << ");\n";
            }
        g.pend.clear();
        g.o << "__syncthreads();\n}\n";
        body << g.o.str();
    }
    if (!g.ok || params.size() * sizeof(R) > kMaxParamBytes) return std::string();
    if (adj) {
        // psi and lambda tiles side by side in shared memory, plain loads and
        // stores; gradient partials in FP64 per CTA, written at the end
        std::ostringstream src;
        src << "#include \"tile_dev.cuh\"\nusing namespace sv;\n"
            << "typedef " << RName<R>::r << " R;\ntypedef " << RName<R>::t << " T;\n"
            << "struct P { R m[" << std::max<size_t>(1, params.size()) << "]; };\n"
            << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", " << RName<R>::minb_adj << ")\n"
            << "svja(T* __restrict__ amps, T* __restrict__ lam, const TileDesc td, const uint64_t gbase, "
               "const uint64_t ntiles, double* __restrict__ gpart, const P p)\n{\n"
            << "extern __shared__ __align__(16) unsigned char smem[];\n"
            << "T* s = reinterpret_cast<T*>(smem);\nT* sl = s + tile::kPadElems;\n"
            << "__shared__ tile::Rows rt;\n__shared__ R gw[" << std::max(1, nslot) * 8 << "];  // [slot][warp]\n"
            << "tile::setup_rows(rt, td);\n" << hoist.str()
            << "for (int k = threadIdx.x; k < " << nslot * 8 << "; k += blockDim.x) gw[k] = (R)0;\n"
            << "const uint32_t bo = 0;\n"
            << "for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {\n__syncthreads();\n"
            << "const uint64_t base = tile::tile_base(rt, td, tl);\n"
            << "tile::load_plain<T, R, tile::PadLayout, " << lrow << ">(s, amps, rt, td, base);\n"
            << "tile::load_plain<T, R, tile::PadLayout, " << lrow << ">(sl, lam, rt, td, base);\n"
            << "__syncthreads();\n"
            << body.str();
        if (!ds)
            src << "tile::store_plain<T, R, tile::PadLayout, " << lrow << ">(s, amps, rt, td, base);\n"
                << "tile::store_plain<T, R, tile::PadLayout, " << lrow << ">(sl, lam, rt, td, base);\n";
        src << "}\n__syncthreads();\n"
            << "for (int k = threadIdx.x; k < " << nslot << "; k += blockDim.x) {\n"
            << "double v = 0.0;\nfor (int w = 0; w < 8; w++) v += (double)gw[k * 8 + w];\n"
            << "gpart[(uint64_t)k * gridDim.x + blockIdx.x] = v;\n}\n"
            << "}\n";
        return src.str();
    }
    const bool pf = prefetches(dec, sizeof(R));
    // rows of the tile: whole codec block pairs (8 low bits) in a sub-pass that
    // decodes or encodes, 16 amplitudes (4 low bits) otherwise
    const std::string lb = std::to_string(lrow);
    std::ostringstream src;
    src << "#include \"tile_dev.cuh\"\nusing namespace sv;\n"
        << "typedef " << RName<R>::r << " R;\ntypedef " << RName<R>::t << " T;\n"
        << "struct P { R m[" << std::max<size_t>(1, params.size()) << "]; };\n"
        << "extern \"C\" __global__ void __launch_bounds__(" << kJitThreads << ", " << RName<R>::minb << ")\n"
        << "svj(T* __restrict__ amps, const TileDesc td, const uint64_t gbase, const uint64_t ntiles, "
           "const FuseArgs fa, const P p)\n{\n"
        << "extern __shared__ __align__(16) unsigned char smem[];\n"
        << "T* s = reinterpret_cast<T*>(smem);\n"
        << "uint32_t* cw = reinterpret_cast<uint32_t*>(smem + sizeof(T) * tile::kPadElems * " << (pf ? 2 : 1) << ");\n"
        << "__shared__ tile::Rows rt;\ntile::setup_rows(rt, td);\n" << hoist.str();
    if (pf) {
        // tile buffer bo (element offset 0 or 4096) is processed while the
        // other one fills; bo is folded into every phase's base offset
        // the next tile's base, computed for its prefetch, is carried over.
        // The copies' offsets are compiled in (the tile's positions are part
        // of the kernel's key): amplitude t + 256k of the tile (t = thread)
        // sits at base + gld + OFF(256k) in HBM and at slot pad(t) + 273k of
        // the buffer (the padded layout and the local offsets are additive
        // over disjoint bits)
        auto sh = [&](int b) { return b < lrow ? b : (int)td.hpos[b - lrow]; };
        std::string gl;
        for (int j = 0; j < 8; j++)
            gl += (j ? " | " : "") + std::string("((uint64_t)((threadIdx.x >> ") + std::to_string(j) + ") & 1u) << " +
                  std::to_string(sh(j)) + ")";
        auto fetch = [&](const std::string& buf, const std::string& bse) {
            std::ostringstream f;
            f << "{ const T* const g = amps + " << bse << " + gld; const uint32_t d = dld + " << sizeof(R) * 2
              << "u * (" << buf << ");\n";
            for (uint32_t k = 0; k < 16; k++) {
                uint64_t off = 0;
                for (int i = 0; i < 4; i++)
                    if ((k >> i) & 1u) off |= 1ull << sh(8 + i);
                f << "asm volatile(\"cp.async.ca.shared.global [%0], [%1], 8;\\n\" :: \"r\"(d + " << sizeof(R) * 2 * 273u * k
                  << "u), \"l\"(g + " << hex(off) << "ull) : \"memory\");\n";
            }
            f << "asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\"); }\n";
            return f.str();
        };
        src << "const uint64_t gld = " << gl << ";\n"
            << "const uint32_t dld = (uint32_t)__cvta_generic_to_shared(s) + " << sizeof(R) * 2
            << "u * (threadIdx.x + (threadIdx.x >> 4));\n"
            << "__syncthreads();\n"
            << "uint64_t base_n = blockIdx.x < ntiles ? tile::tile_base(rt, td, blockIdx.x) : 0ull;\n"
            << "if (blockIdx.x < ntiles) " << fetch("0u", "base_n")
            << "uint32_t bo = 0;\n"
            << "for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, bo = tile::kPadElems - bo) {\n"
            << "const uint64_t base = base_n;\n"
            << "tile::cp_async_wait_all();\n__syncthreads();\n"
            << "if (tl + gridDim.x < ntiles) {\nbase_n = tile::tile_base(rt, td, tl + gridDim.x);\n"
            << fetch("tile::kPadElems - bo", "base_n") << "}\n";
    } else {
        src << "const uint32_t bo = 0;\n"
            << "for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {\n__syncthreads();\n"
            << "const uint64_t base = tile::tile_base(rt, td, tl);\n"
            << "tile::load_tile<T, R, " << (dec ? "true" : "false") << ", tile::PadLayout, " << lb
            << ">(s, amps, rt, td, base, fa, cw);\n"
            << "__syncthreads();\n";
    }
    src << body.str();
    if (!ds)
        src << "tile::store_tile<T, R, " << (enc ? "true" : "false") << ", tile::PadLayout, " << lb
            << ">(s + bo, amps, rt, td, base, fa, cw);\n";
    src << "}\n}\n";
    return src.str();
}

bool jit_compile(const std::vector<std::string>& keys, const std::function<std::string(size_t)>& source_of,
                 int device, std::vector<const JitFn*>& fns, std::string& err, JitReport* rep)
{
    const auto t0 = std::chrono::steady_clock::now();
    fns.assign(keys.size(), nullptr);
    std::lock_guard<std::mutex> lk(g_mu);
    Drv& d = drv();
    if (!d.ok) {
        err = d.why;
        return false;
    }
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
        err = "cannot query the device's compute capability";
        return false;
    }
    const std::string arch = "sm_" + std::to_string(major * 10 + minor) + (major >= 9 ? "a" : "");
    const std::string prefix = std::to_string(device) + "/" + arch + "/";
    std::vector<Job> jobs;
    std::vector<std::string> srcs;
    std::unordered_map<std::string, size_t> job_of;
    for (size_t i = 0; i < keys.size(); i++) {
        if (keys[i].empty()) continue;
        std::string key = prefix + keys[i];
        if (g_cache.count(key) || job_of.count(key)) continue;
        job_of[key] = jobs.size();
        Job j;
        j.index = i;
        j.key = std::move(key);
        jobs.push_back(std::move(j));
    }
    // sources of the kernels not compiled yet (an empty source: the sub-pass
    // cannot be specialised and stays on the table-driven kernel)
    srcs.resize(jobs.size());
    std::vector<Job*> todo;
    for (size_t k = 0; k < jobs.size(); k++) {
        srcs[k] = source_of(jobs[k].index);
        jobs[k].src = &srcs[k];
        if (!srcs[k].empty()) todo.push_back(&jobs[k]);
    }
    if (!todo.empty()) {
        Nvrtc& n = nvrtc();
        if (!n.ok) {
            err = n.why;
            return false;
        }
        const std::string arch_opt = "--gpu-architecture=" + arch;
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const size_t nthr = std::min<size_t>(todo.size(), hw);
        std::vector<std::thread> pool;
        std::atomic_size_t next{0};
        for (size_t t = 0; t < nthr; t++)
            pool.emplace_back([&]() {
                for (size_t k; (k = next.fetch_add(1)) < todo.size();) compile_one(*todo[k], arch_opt);
            });
        for (std::thread& th : pool) th.join();
        if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
            err = "cannot make the device current";
            return false;
        }
    }
    const size_t tile_bytes = sizeof(double) * 2 * tile_pad_elems();
    const int smem_max = (int)std::max(tile_bytes + sizeof(uint32_t) * 2 * 264 * (kJitThreads / 32), 2 * tile_bytes);
    for (Job& j : jobs) {
        auto fn = std::make_unique<JitFn>();
        fn->lrow = (uint8_t)j.key[prefix.size() + kKeyHeader - 1];
        if (!j.src->empty()) {
            if (!j.ok) {
                err = "NVRTC compilation failed: " + j.log.substr(0, 2000);
                return false;
            }
            CUresult r = d.load(&fn->mod, j.cubin.data());
            if (r == CUDA_SUCCESS) {
                // svj: a sub-pass kernel; svja: an adjoint (two-vector) one
                r = d.getfn(&fn->fn, fn->mod, j.src->find("\nsvja(") != std::string::npos ? "svja" : "svj");
            }
            if (r == CUDA_SUCCESS) r = d.setattr(fn->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem_max);
            if (r != CUDA_SUCCESS) {
                err = "loading a compiled kernel failed (CUresult " + std::to_string((int)r) + ")";
                return false;
            }
            if (rep) rep->compiled++;
        }
        g_cache[j.key] = std::move(fn);
    }
    for (size_t i = 0; i < keys.size(); i++) {
        if (keys[i].empty()) continue;
        const JitFn* f = g_cache[prefix + keys[i]].get();
        fns[i] = f->fn ? f : nullptr;
    }
    if (rep) rep->seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

unsigned jit_grid(uint64_t ntiles) { return (unsigned)std::min<uint64_t>(ntiles, 152ull * 32); }

template <typename R>
cudaError_t jit_launch_adjoint(const JitFn* fn, void* psi, void* lam, const TileDesc& td, uint64_t gbase,
                               double* gpart, const std::vector<R>& params, cudaStream_t st, unsigned* grid_out)
{
    if (!fn || td.t != kPhaseTileQubits || td.l != fn->lrow || params.empty()) return cudaErrorInvalidValue;
    const uint64_t ntiles = 1ull << (td.L - kPhaseTileQubits);
    const unsigned grid = jit_grid(ntiles);
    if (grid_out) *grid_out = grid;
    const size_t smem = sizeof(R) * 2 * tile_pad_elems() * 2;
    void* a = psi;
    void* b = lam;
    TileDesc t = td;
    uint64_t gb = gbase, nt = ntiles;
    double* gp = gpart;
    void* args[] = {&a, &b, &t, &gb, &nt, &gp, const_cast<R*>(params.data())};
    const CUresult r = drv().launch(fn->fn, grid, 1, 1, kJitThreads, 1, 1, (unsigned)smem, (CUstream)st, args, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

template <typename R>
cudaError_t jit_launch(const JitFn* fn, void* amps, const TileDesc& td, uint64_t gbase, const FuseArgs& fa,
                       const std::vector<R>& params, cudaStream_t st)
{
    // the kernel was generated for the tile rows of its sub-pass (8 low bits when it decodes or encodes)
    if (!fn || td.t != kPhaseTileQubits || td.l != fn->lrow || params.empty()) return cudaErrorInvalidValue;
    const uint64_t ntiles = 1ull << (td.L - kPhaseTileQubits);
    const unsigned grid = jit_grid(ntiles);
    const size_t smem = (sizeof(R) * 2 * tile_pad_elems() * (prefetches(fa.decode != 0, sizeof(R)) ? 2 : 1)) +
                        ((fa.decode || fa.encode) ? sizeof(uint32_t) * 2 * 264 * (kJitThreads / 32) : 0);
    void* a = amps;
    TileDesc t = td;
    uint64_t gb = gbase, nt = ntiles;
    FuseArgs f = fa;
    void* args[] = {&a, &t, &gb, &nt, &f, const_cast<R*>(params.data())};
    const CUresult r = drv().launch(fn->fn, grid, 1, 1, kJitThreads, 1, 1, (unsigned)smem, (CUstream)st, args, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

template void jit_params<float>(const Phase*, int, const PhaseOp<float>*, const float*, std::vector<float>&, bool);
template void jit_params<double>(const Phase*, int, const PhaseOp<double>*, const double*, std::vector<double>&,
                                 bool);
template void jit_key<float>(const Phase*, int, const PhaseOp<float>*, const CtaCtrl*, const std::vector<float>&,
                             bool, bool, const TileDesc&, std::string&, const int32_t*);
template void jit_key<double>(const Phase*, int, const PhaseOp<double>*, const CtaCtrl*, const std::vector<double>&,
                              bool, bool, const TileDesc&, std::string&, const int32_t*);
template std::string jit_source<float>(const Phase*, int, const PhaseOp<float>*, const CtaCtrl*, const float*, bool,
                                       bool, const TileDesc&, const std::vector<float>&, const int32_t*);
template std::string jit_source<double>(const Phase*, int, const PhaseOp<double>*, const CtaCtrl*, const double*,
                                        bool, bool, const TileDesc&, const std::vector<double>&, const int32_t*);
template cudaError_t jit_launch<float>(const JitFn*, void*, const TileDesc&, uint64_t, const FuseArgs&,
                                       const std::vector<float>&, cudaStream_t);
template cudaError_t jit_launch_adjoint<float>(const JitFn*, void*, void*, const TileDesc&, uint64_t, double*,
                                               const std::vector<float>&, cudaStream_t, unsigned*);
template cudaError_t jit_launch_adjoint<double>(const JitFn*, void*, void*, const TileDesc&, uint64_t, double*,
                                                const std::vector<double>&, cudaStream_t, unsigned*);
template cudaError_t jit_launch<double>(const JitFn*, void*, const TileDesc&, uint64_t, const FuseArgs&,
                                        const std::vector<double>&, cudaStream_t);

}  // namespace sv
