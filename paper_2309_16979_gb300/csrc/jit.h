// jit.h -- sub-pass kernels specialised to their gate sequence, generated at
// run time and compiled with NVRTC (jit.cpp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "sv_internal.h"

namespace sv {

struct JitFn;  // a loaded kernel (owned by the process-wide cache)

// The kernel for one register-phase sub-pass is described by its phases and
// ops as dev_phases lays them out, whether it decodes the chunk streams (dec),
// whether it encodes the block pairs (enc), and its tile (td: the low bits
// of its rows, td.l, 4, or 8 with the codec; where the last phase stores
// straight to HBM, the positions of the tile's other bits, td.hpos).
//
// jit_params: the kernel's by-value parameter block, the matrix values of its
// ops in order, 8 per op (32 for a 4x4). Ops that act on every amplitude are
// stored divided by their largest-magnitude entry, and the product of those
// scalars is multiplied into the last of them, so the sub-pass's result is
// unchanged while most gates carry an exact 1.
template <typename R>
void jit_params(const Phase* ph, int nph, const PhaseOp<R>* ops, const R* d2m, std::vector<R>& params,
                bool factor = true);

// jit_key: a compact description of everything the generated code depends
// on (the sub-pass's structure and which entries of `params` are exactly 0,
// +-1, +-i or equal to each other), not on the remaining values.
template <typename R>
void jit_key(const Phase* ph, int nph, const PhaseOp<R>* ops, const CtaCtrl* ctl, const std::vector<R>& params,
             bool dec, bool enc, const TileDesc& td, std::string& key, const int32_t* grad = nullptr);

// jit_source: the CUDA C++ source of the kernel, reading `params`. Empty when
// the sub-pass cannot be specialised (it then runs on the table-driven kernel).
//
// Adjoint sub-passes (MEMQSim has none; the reverse sweep of the adjoint
// method) pass `grad` (dev_phases' per-op gradient slots) and no codec: the
// kernel applies every op to psi and to lambda, and before each
// parameterised op adds Im<lambda| G |psi> of its tiles to a per-CTA FP64
// partial, written to gpart[slot * gridDim.x + blockIdx.x]; `params` is then
// built with factor = false (a scalar factored out would scale the partials).
template <typename R>
std::string jit_source(const Phase* ph, int nph, const PhaseOp<R>* ops, const CtaCtrl* ctl, const R* d2m, bool dec,
                       bool enc, const TileDesc& td, const std::vector<R>& params, const int32_t* grad = nullptr);

// Look the kernels of `keys` up in the process-wide cache for `device`;
// generate (source_of(i)), compile (in parallel) and load the ones missing.
// fns[i] receives the kernel of keys[i], nullptr for an empty key or an
// unspecialisable sub-pass. On failure returns false with the reason in `err`.
struct JitReport {
    uint64_t compiled = 0;   // kernels compiled by this call
    double seconds = 0;      // wall time spent looking up, generating, compiling and loading
};
bool jit_compile(const std::vector<std::string>& keys, const std::function<std::string(size_t)>& source_of,
                 int device, std::vector<const JitFn*>& fns, std::string& err, JitReport* rep);

// Launch a generated kernel over the 2^(td.L - 12) tiles of `amps`.
template <typename R>
cudaError_t jit_launch(const JitFn* fn, void* amps, const TileDesc& td, uint64_t gbase, const FuseArgs& fa,
                       const std::vector<R>& params, cudaStream_t st);

// Launch a generated adjoint kernel over the tiles of psi and lambda; *grid
// receives the number of CTAs (the stride of its gradient partials).
template <typename R>
cudaError_t jit_launch_adjoint(const JitFn* fn, void* psi, void* lam, const TileDesc& td, uint64_t gbase,
                               double* gpart, const std::vector<R>& params, cudaStream_t st, unsigned* grid);

// CTAs of a generated kernel's launch over `ntiles` tiles.
unsigned jit_grid(uint64_t ntiles);

}  // namespace sv
