// sv_dev_types.h -- plain types shared by the device code of the library
// and by the sub-pass kernels generated at run time (jit.cpp), which compile
// this header with NVRTC; it therefore includes no system header there.
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>
#endif

namespace sv {

// ------------------------------------------------------------------ codec
constexpr uint32_t kMagic = 0x31435653u;  // "SVC1"
constexpr int kBlock = 256;               // values per codec block

struct CodecLayout {
    uint32_t nb;      // blocks, both planes
    uint32_t bpc;     // block pairs (256 amplitudes each) per chunk
    size_t w_off, a_off, o_off, p_off;
    size_t max_bytes; // metadata + worst-case payload (32 bits per value)
};

__host__ __device__ inline size_t pad16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline CodecLayout codec_layout(int c)
{
    CodecLayout L;
    L.nb = (uint32_t)((2ull << c) >> 8);
    L.bpc = L.nb / 2;
    L.w_off = 32;
    L.a_off = L.w_off + pad16(L.nb);
    L.o_off = L.a_off + pad16(4ull * L.nb);
    L.p_off = L.o_off + pad16(4ull * (L.nb + 1));
    L.max_bytes = L.p_off + (size_t)L.nb * 1024;
    return L;
}

// device -> host record of one encoded chunk
struct ChunkOut {
    uint64_t bytes;   // stream length
    uint64_t sumsq;   // sum of q^2 over the chunk (exact; norm^2 = sumsq * Delta^2)
    int32_t k;        // the chunk's step exponent, Delta = 2^k
    int32_t pad;
};

// kErrWait: a kernel gave up waiting for its own asynchronous copies (an
// iteration limit on every spin-wait) and skipped the rest of its work
enum : int { kErrCorrupt = 1, kErrRange = 2, kErrWait = 4 };

// Register-phase form of a sub-pass (tiles of exactly kPhaseTileQubits
// qubits, 256 threads, 16 amplitudes per thread): a phase keeps 4 tile
// qubits in registers and applies every op whose mixing qubits are among
// them; phases exchange amplitudes through shared memory.
constexpr int kPhaseTileQubits = 12;
constexpr int kPhaseRegBits = 4;
// Local qubits 0..3 are in every tile: a tile is 256 rows of 16 contiguous
// amplitudes (128 B of complex64, one full line per row), which leaves 8 of
// the 12 tile qubits to the planner. Sub-passes that fuse the codec take
// rows of 256 (whole block pairs).
constexpr int kTileLowQubits = 4;

constexpr int kMaxTileQubits = 13;
constexpr int kMaxLocalQubits = 48;

struct TileDesc {
    int32_t t;                  // tile qubits
    int32_t l;                  // low local bits 0..l-1 always in the tile (rows are 2^l contiguous)
    int32_t L;                  // local qubits of the buffer (c + g, or n when uncompressed)
    int32_t nout;               // L - t
    int8_t hpos[kMaxTileQubits];          // local positions of tile bits l..t-1
    int8_t opos[kMaxLocalQubits];         // local positions outside the tile (ascending)
};

// per-group staging parameters for decode
constexpr int kMaxGroupChunks = 256;

struct GroupIn {
    uint32_t bytes[kMaxGroupChunks];      // stream length of each staged chunk
};

// Optional fusion of the chunk codec into a tile sub-pass (tiles whose rows
// are whole 256-amplitude block pairs, i.e. l = 8): decode the group's chunk
// streams straight into shared memory instead of reading amplitudes, and/or
// encode the tile's block pairs (widths, anchors, packed staging, sum q^2)
// instead of writing amplitudes; launch_encode_finish then completes the
// streams (offset scan, header, compaction).
struct FuseArgs {
    int32_t decode = 0, encode = 0;
    int32_t c = 0, dtype = 0, k = 0;
    double scale = 1.0;
    const uint8_t* in = nullptr;
    size_t in_stride = 0;
    GroupIn gin{};
    uint8_t* out = nullptr;
    size_t out_stride = 0;
    uint32_t* sparse = nullptr;
    unsigned long long* blocksq = nullptr;
    int* err = nullptr;
};

}  // namespace sv
