// engine.h -- pass execution entry points used by the C ABI (api.cpp).
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include "runtime.h"

namespace sv {

// Device memory of a handle: the caller's provider (sv_config.device_alloc /
// device_free) when set, else cudaMalloc / cudaFree. dev_free(s, nullptr) is a no-op.
template <typename T>
cudaError_t dev_alloc(sv_state* s, T** p, size_t bytes)
{
    if (!s->cfg.device_alloc) return cudaMalloc(p, bytes);
    void* q = s->cfg.device_alloc(std::max<size_t>(1, bytes), s->cfg.device, s->cfg.alloc_ctx);
    *p = static_cast<T*>(q);
    return q ? cudaSuccess : cudaErrorMemoryAllocation;
}
inline void dev_free(sv_state* s, void* p)
{
    if (!p) return;
    if (s->cfg.device_free) s->cfg.device_free(p, s->cfg.device, s->cfg.alloc_ctx);
    else cudaFree(p);
}

int fail(sv_state* s, int code, const std::string& msg);
int cuda_fail(sv_state* s, cudaError_t e, const char* where);
int wait_stream(sv_state* s, cudaStream_t st);
int sync_all(sv_state* s);
int check_device_error(sv_state* s);
// Destination of a chunk stream of `bytes` bytes: the chunk's own slot when
// the stream fits (rewritten in place), else a larger slot with 1/32 headroom
// (the old slot is released to the pool for reuse). ref is updated; nullptr
// when pinned memory (or the host budget) is exhausted. Callers write the
// slot only after every reader of the chunk's previous stream has finished.
uint8_t* store_slot(sv_state* s, HostPool& pool, ChunkRef& ref, uint64_t bytes);
// Return every chunk's slot to the pool (no copy may still read or write them).
void store_release_all(HostPool& pool, std::vector<ChunkRef>& refs);
void pool_free(HostPool& pool);
void tile_shape(int L, int tq, int lq, int& t, int& l);

template <typename R> int init_state(sv_state* s);
// remap: move qubits between high and low positions when that saves passes
// (plan_circuit); s->perm follows.
template <typename R> int apply_circuit(sv_state* s, const std::vector<PGate>& gates, bool remap);
// host only: the sources of the kernels apply_circuit would generate
template <typename R>
int jit_sources(sv_state* s, const std::vector<PGate>& gates, std::vector<std::string>& out, bool adjoint);
template <typename R> int amplitudes(sv_state* s, const uint64_t* idx, size_t m, double* out);
// out[0] + i out[1] = <a|b>; b uncompressed on a's device, same n
template <typename RA, typename RB> int inner(sv_state* a, const sv_state* b, double* out);
template <typename R> int expect(sv_state* s, const sv_pauli_term* terms, size_t nterms, double* out_re);
template <typename R>
int grad_compressed(sv_state* s, const std::vector<PGate>& gates, size_t nparams, const sv_pauli_term* H,
                    size_t nterms, double* energy, double* grad);
template <typename R>
int grad_uncompressed(sv_state* s, const std::vector<PGate>& gates, size_t nparams, const sv_pauli_term* H,
                      size_t nterms, double* energy, double* grad);

}  // namespace sv
