// jit.h -- sub-pass kernels specialised to their gate sequence, generated at
// run time and compiled with NVRTC (jit.cpp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sv_internal.h"

namespace sv {

struct JitFn;  // a loaded kernel (owned by the process-wide cache)

// CUDA C++ source of the kernel for one register-phase sub-pass: its phases
// and ops (as dev_phases lays them out), whether it decodes the chunk streams
// (dec) and/or encodes the block pairs (enc). The matrix values the kernel
// reads are appended to `params` (the kernel's by-value parameter block); the
// source depends only on the sub-pass's structure, not on those values.
// Returns an empty string when the sub-pass cannot be specialised (it then
// runs on the table-driven kernel).
template <typename R>
std::string jit_source(const Phase* ph, int nph, const PhaseOp<R>* ops, const CtaCtrl* ctl, const R* d2m, bool dec,
                       bool enc, std::vector<R>& params);

// Compile (in parallel) and load the kernels of `sources` for `device`,
// reusing kernels compiled before in this process; fns[i] receives the
// kernel of sources[i] (nullptr for an empty source). On failure returns
// false with the reason in `err`.
struct JitReport {
    uint64_t compiled = 0;   // kernels compiled by this call
    double seconds = 0;      // wall time spent compiling and loading
};
bool jit_compile(const std::vector<std::string>& sources, int device, std::vector<const JitFn*>& fns,
                 std::string& err, JitReport* rep);

// Launch a generated kernel over the 2^(td.L - 12) tiles of `amps`.
template <typename R>
cudaError_t jit_launch(const JitFn* fn, void* amps, const TileDesc& td, uint64_t gbase, const FuseArgs& fa,
                       const std::vector<R>& params, cudaStream_t st);

}  // namespace sv
