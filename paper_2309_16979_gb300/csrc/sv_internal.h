// sv_internal.h -- types shared by the CUDA kernels and the host runtime.
//
// Terminology (MEMQSim, Sec. 2): the state vector is split into chunks of
// 2^c amplitudes; a pass ("stage") streams every chunk through the GPU once.
// A pass stages groups of 2^g chunks that differ only in the pass's staged
// high qubits S, so that gates mixing those qubits act inside one group. In a
// group, the local index of an amplitude is (slot << c) | low bits; local
// qubit positions are 0..c-1 for the low qubits and c..c+g-1 for S.
// Inside a group, a tile is the 2^t amplitudes that vary over t local
// positions T with all other local bits fixed; a sub-pass sweeps every tile
// of a group once, applying all of its gates in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sv_dev_types.h"

namespace sv {

// --------------------------------------------------------------- gate ops
enum OpType : int32_t { OP_DENSE1 = 0, OP_DENSE2 = 1, OP_DIAG = 2 };

// A bit source of a diagonal gate's index: tile-local bit, local bit outside
// the tile, or a global (fixed per group) bit.
enum : int32_t { SRC_NONE = -1, SRC_TILE = 0, SRC_LOCAL = 64, SRC_GLOBAL = 128 };

template <typename R>
struct DevOp {
    int32_t type;          // OpType
    int32_t t0, t1;        // tile-local bit positions of dense targets
    int32_t d0, d1;        // diagonal entry-index bit sources (SRC_* + position)
    uint32_t cmask_tile;   // controls on tile-local bits
    uint64_t cmask_local;  // controls on local bits outside the tile
    uint64_t cmask_global; // controls on global bits fixed per group
    int32_t grad_slot;     // adjoint: >= 0 -> gradient term taken before this op
    int32_t gen;           // adjoint generator on t0 / d0: 1 = X, 2 = Y, 3 = Z
    R m[32];               // dense1: 2x2, dense2: 4x4, diag: 4 entries; (re, im) pairs
};

// Op kinds of a phase. A phase op's `code` is dense, so one jump-table
// dispatch selects code specialised at compile time:
//   kinds PK_GENERIC..PK_DIAG1 (one register bit b0): code = kind * 8 + ctrl * 4 + b0
//   PK_DIAG2 (register bits b0, b1):                  code = 40 + ctrl * 16 + b1 * 4 + b0
//   PK_DIAGT:                                          code = 72 + ctrl
//   PK_DENSE2 (register bits b0, b1):                  code = 74, bits in `pad` (b1 * 4 + b0)
// where ctrl says the op has controls among the register bits.
enum PhaseOpKind : uint32_t {
    PK_GENERIC = 0,  // 2x2 complex matrix on register bit b0
    PK_REAL = 1,     // 2x2 real matrix
    PK_RX = 2,       // [[p, i q], [i r, s]] with real p, q, r, s
    PK_UNUSED3 = 3,  // (free: an exchange form for X measured slower than X as a real matrix)
    PK_DIAG1 = 4,    // diagonal whose entry index has one register bit b0
    PK_DIAG2 = 5,    // diagonal whose entry index bits are register bits (b0, b1)
    PK_DIAGT = 6,    // diagonal whose entry index is constant per thread
    PK_DENSE2 = 7    // 4x4 complex matrix on register bits (b0, b1), matrix in a side table
};
constexpr uint32_t kCodeDiag2 = 40, kCodeDiagT = 72, kCodeDense2 = 74;
// A constant bit source byte: 0xff none, 0..15 tile bit (a thread bit in the
// phase), 0x40 + p local bit p outside the tile, 0x80 + q global bit q.
constexpr uint8_t kSrcNone = 0xff;

template <typename R>
struct PhaseOp {
    uint16_t code;
    uint16_t amask;  // register controls: bit i set = register index i takes part
    uint16_t tmask;  // controls on thread (non-register tile) bits
    uint8_t flags;   // bit 0: controls outside the tile, entry `aux` of the CTA control table
    uint8_t csrc;    // PK_DIAG1: source of the entry-index bit that is not the register bit;
                     // PK_DIAGT: source of entry-index bit 0
    uint8_t csrc1;   // PK_DIAGT: source of entry-index bit 1
    uint8_t rsel;    // PK_DIAG1: which entry-index bit (0 or 1) is the register bit
    uint16_t pad;
    uint32_t aux;    // CTA control table entry / PK_DENSE2 matrix index
    R m[8];          // 2x2 matrix or 4 diagonal entries, (re, im) pairs
};

struct CtaCtrl {
    uint64_t cl;  // local bits outside the tile that must be 1
    uint64_t cg;  // global bits (fixed per group) that must be 1
};

struct Phase {
    uint16_t sroff[1 << kPhaseRegBits];                  // swizzled tile offset of register index m
    int32_t op_begin, op_count;
    int8_t rpos[kPhaseRegBits];                          // register bit j <-> tile bit rpos[j]
    int8_t tpos[kPhaseTileQubits - kPhaseRegBits];       // thread bit j <-> tile bit tpos[j]
    uint32_t pad[3];
};
static_assert(sizeof(Phase) == 64, "phase records are 64 bytes");

// ------------------------------------------------------------ launchers
// All launchers enqueue on `st` and return cudaGetLastError().

template <typename R>
cudaError_t launch_decode(const uint8_t* in, size_t stride, int c, int dtype, int nchunks,
                          const GroupIn& gin, void* amps, double scale, int* err, cudaStream_t st);

template <typename R>
cudaError_t launch_encode(const void* amps, int c, int dtype, int k, int nchunks, uint8_t* out,
                          size_t stride, uint32_t* sparse, unsigned long long* blocksq,
                          ChunkOut* chunk_out, int* err, cudaStream_t st, int* launches,
                          const int32_t* kc = nullptr);

// Relative bound: per-chunk step exponents kc[0..nchunks) of the chunks at
// amps (2^c amplitudes each) from their largest component (mbits: scratch).
// launch_encode with kc != nullptr encodes chunk r with step 2^kc[r].
template <typename R>
cudaError_t launch_chunk_steps(const void* amps, int c, int nchunks, double eb, unsigned long long* mbits,
                               int32_t* kc, cudaStream_t st, int* launches);

template <typename R>
cudaError_t launch_apply(void* amps, const TileDesc& td, const DevOp<R>* ops, int nops,
                         uint64_t gbase, cudaStream_t st);

// Capacity of the constant-memory phase / op tables (one pass at a time).
constexpr int kConstPhases = 128;
constexpr int kConstOpsF = 640;
constexpr int kConstOpsD = 256;

// Copy a pass's phase and op tables to constant memory (stream-ordered);
// returns false (nothing copied) when they do not fit.
template <typename R>
bool upload_const_tables(const Phase* phases, int nphases, const PhaseOp<R>* ops, int nops, cudaStream_t st);

// ph_base >= 0: the sub-pass's phases start at c_phases[ph_base] and its ops
// are read from the constant op table (upload_const_tables); otherwise from
// `phases` / `ops` in device memory.
template <typename R>
cudaError_t launch_apply_phases(void* amps, const TileDesc& td, const Phase* phases, int nphases,
                                const PhaseOp<R>* ops, int op0, int nops, const CtaCtrl* ctl, const R* dense2,
                                uint64_t gbase, const FuseArgs& fa, cudaStream_t st, int ph_base = -1);

cudaError_t launch_encode_finish(int c, int dtype, int k, int nchunks, uint8_t* out, size_t stride,
                                 const uint32_t* sparse, const unsigned long long* blocksq, ChunkOut* chunk_out,
                                 cudaStream_t st, int* launches, const int32_t* kc = nullptr);

template <typename R>
cudaError_t launch_fill_basis(void* amps, uint64_t count, int64_t one_at, cudaStream_t st);

// Stream copies between the device slots of consecutive passes: the first
// co[j].bytes bytes of stream j (at j * stride in src) to the same place in
// dst, its length to bytes[j]; and streams mv.src[i] of src (lengths from
// bytes) to slots mv.dst[i] of dst.
struct StreamMoves {
    uint16_t src[kMaxGroupChunks];
    uint16_t dst[kMaxGroupChunks];
    int32_t n = 0;
};
cudaError_t launch_copy_streams(const uint8_t* src, const ChunkOut* co, uint8_t* dst, uint64_t* bytes, size_t stride,
                                int n, cudaStream_t st);
// stream mv.src[i] (at src + mv.src[i] * src_stride, bytes[mv.src[i]] long)
// -> dst + mv.dst[i] * dst_stride
cudaError_t launch_gather_streams(const uint8_t* src, const uint64_t* bytes, size_t src_stride, uint8_t* dst,
                                  size_t dst_stride, const StreamMoves& mv, cudaStream_t st);

// sum_t coeff_t <A| P_t |B> pieces; see reduce.cu
struct PauliDev {
    double coeff;
    uint64_t xl;      // x-mask on the buffer's local bits
    uint64_t zl;      // z-mask on local bits
    uint64_t zg;      // z-mask on global bits fixed per unit (phase sign)
    int32_t ny;       // number of Y factors mod 4
    int32_t pad;
};

template <typename R>
cudaError_t launch_pauli_partials(const void* A, const void* B, int Lbits, uint64_t gbase,
                                  const PauliDev* terms, int nterms, double* partials, int nblocks,
                                  cudaStream_t st);

// partials[0..nblocks) = per-CTA shares of <psi|H|psi> over a 2^Lbits buffer
// for all nterms terms (at most max_energy_terms()) in one sweep
template <typename R>
cudaError_t launch_energy_partials(const void* psi, int Lbits, uint64_t gbase, const PauliDev* terms, int nterms,
                                   double* partials, int nblocks, cudaStream_t st);
int max_energy_terms();

cudaError_t launch_sum_partials(const double* partials, int nterms, int nblocks, double* out,
                                cudaStream_t st);

// Tiles of 4096 amplitudes of a 2^Lbits buffer for k_energy_tiles: local bits
// 0..7 and the four local positions hp[0..3] (all >= 8); op[0..nout) are the
// other positions, ascending (the tile index's bits, low first).
struct EnergyTiles {
    int8_t hp[4];
    int8_t op[kMaxLocalQubits];
    int32_t nout;
};
constexpr int kEnergyTileBits = 12;

// partials[0..nblocks) = per-CTA shares of sum_t <psi|P_t|psi> over the
// buffer for terms whose x-masks lie in the tiles' bits (at most
// max_energy_terms()); partners read from the tile in shared memory, tiles
// brought in by bulk copies. psi must be 16-byte aligned. A wait for the
// copies that exceeds its limit sets kErrWait in *err.
template <typename R>
cudaError_t launch_energy_tiles(const void* psi, int Lbits, uint64_t gbase, const EnergyTiles& et,
                                const PauliDev* terms, int nterms, double* partials, int nblocks, int* err,
                                cudaStream_t st);

template <typename R>
cudaError_t launch_gather(const void* amps, const uint64_t* local_idx, const uint64_t* dest,
                          uint64_t m, double* out, cudaStream_t st);

template <typename R>
cudaError_t launch_hamiltonian(const void* psi, void* lam, int n, const PauliDev* terms, int nterms,
                               cudaStream_t st);

template <typename R>
cudaError_t launch_adjoint(void* psi, void* lam, const TileDesc& td, const DevOp<R>* ops, int nops,
                           uint64_t gbase, double* gpart, uint64_t tile_stride, cudaStream_t st);

// lam (+)= sum_t coeff_t P_t psi over one output chunk of 2^c amplitudes from
// staged source slots (term t reads slot terms[t].pad); accumulate: add to lam
template <typename R>
cudaError_t launch_ham_chunk(const void* psi_slots, void* lam, int c, const PauliDev* terms, int nterms,
                             bool accumulate, cudaStream_t st);

template <typename R>
cudaError_t launch_dot(const void* A, const void* B, uint64_t count, double* partials,
                       int nblocks, cudaStream_t st);

int reduce_blocks_for(uint64_t count);

// Where the amplitudes of one state sit in another: physical index bit j of
// the first is bit pos[j] of the second (identity: the same index).
struct IndexMap {
    int32_t n = 0;
    int32_t identity = 1;
    int8_t pos[64] = {};
};

// partials[0 * nblocks + b], partials[1 * nblocks + b] = Re, Im of CTA b's
// share of sum_i conj(A[i]) * B[map(base + i)], i < count, in FP64; A and B
// may differ in precision (RA, RB).
template <typename RA, typename RB>
cudaError_t launch_inner(const void* A, uint64_t count, uint64_t base, const void* B, const IndexMap& map,
                         double* partials, int nblocks, cudaStream_t st);

}  // namespace sv
