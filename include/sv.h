/*
 * sv.h -- C ABI of the GB300 compressed state-vector simulator.
 *
 * Method: MEMQSim (arXiv 2309.16979). The n-qubit state vector is split into
 * 2^(n-c) chunks of 2^c amplitudes; each chunk is compressed independently
 * and stored in host memory (Sec. 2, "Offline stage"). Each pass over the
 * circuit streams chunks to the GPU, updates them there and stores them back
 * recompressed (Sec. 2, "Online stage", steps (1)-(4) and (6)); whole chunks
 * are moved with bulk copies and placed by GPU threads (Sec. 2, second
 * data-movement strategy; Table 1 "Buffer copy").
 *
 * In this library decompression and recompression run on the GPU, chunks
 * move compressed over the host link, and every step of a pass runs in this
 * library's CUDA kernels (sm_103a).
 *
 * Conventions for every call:
 *   - Qubit 0 is the least-significant bit of an amplitude index.
 *   - Return value 0 (SV_OK) on success, a negative SV_ERR_* code otherwise;
 *     nothing is thrown across the ABI. sv_last_error() describes the last
 *     failure on a handle.
 *   - Every call is synchronous: when it returns, all GPU work it issued has
 *     finished and every output buffer is written.
 *   - Pointers named h_* are host memory, d_* device memory of the handle's
 *     GPU. Inputs are read during the call only; the caller keeps ownership.
 *   - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef SV_GB300_SV_H
#define SV_GB300_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SV_OK 0
#define SV_ERR_ARG (-1)           /* invalid argument (qubit out of range, bad gate, ...) */
#define SV_ERR_HOST_OOM (-2)      /* pinned host allocation failed or host budget exceeded */
#define SV_ERR_DEVICE_OOM (-3)    /* device allocation failed or device budget too small */
#define SV_ERR_CORRUPT (-4)       /* a compressed chunk stream failed validation */
#define SV_ERR_TIMEOUT (-5)       /* a host wait on GPU work exceeded sv_config.timeout_s */
#define SV_ERR_NORM_COLLAPSE (-6) /* norm^2 of the stored state fell below 1e-300 */
#define SV_ERR_RANGE (-7)         /* a value is outside the quantiser's range (or not finite) */
#define SV_ERR_CUDA (-8)          /* a CUDA runtime call failed */

/* ------------------------------------------------------------- enumerations */
enum sv_dtype { SV_C64 = 1, SV_C128 = 2 };       /* amplitude type: complex64 / complex128 */
enum sv_mode { SV_COMPRESSED = 0, SV_UNCOMPRESSED = 1 };

enum sv_gate_kind {
    SV_GATE_H = 0, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_S, SV_GATE_SDG, SV_GATE_T,
    SV_GATE_TDG, SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ, SV_GATE_P, SV_GATE_CNOT, SV_GATE_CZ,
    SV_GATE_CP, SV_GATE_SWAP, SV_GATE_CUSTOM
};

/*
 * One gate. RX/RY/RZ(theta) = exp(-i theta {X,Y,Z} / 2); P(theta) and
 * CP(theta) = diag(1, e^{i theta}) on the target; CNOT/CZ/CP need at least
 * one control; any kind may carry up to 2 controls (the gate acts where all
 * controls are 1). SWAP and 2-target CUSTOM use targets[0..1]; the matrix
 * row/column index has bit b <-> targets[b]. CUSTOM: mat holds the row-major
 * 2^ntargets x 2^ntargets complex matrix as (re, im) pairs; it must be unitary
 * for the error bound of the stored state to mean anything.
 * param_index >= 0 marks a trainable angle for sv_grad (uncontrolled RX, RY or
 * RZ only); other calls use theta and ignore param_index.
 */
typedef struct sv_gate {
    uint32_t kind;
    uint32_t ntargets;
    uint32_t ncontrols;
    int32_t param_index;
    uint32_t targets[2];
    uint32_t controls[2];
    double theta;
    double mat[32];
} sv_gate;

/* coeff * prod_q sigma_q with sigma = I, X (x bit), Z (z bit), Y (both bits). */
typedef struct sv_pauli_term {
    double coeff;
    uint64_t xmask;
    uint64_t zmask;
} sv_pauli_term;

/*
 * Device memory provider for a handle (sv_config.device_alloc / device_free):
 * alloc returns `bytes` of device memory on `device` (NULL on failure, which
 * the calling entry point reports as SV_ERR_DEVICE_OOM); free returns memory
 * that alloc gave. Both are called on the thread that called the library,
 * with `ctx` = sv_config.alloc_ctx. The library frees a block only after all
 * of its own GPU work that uses the block has completed, so a caching
 * allocator may hand the block out again at once.
 */
typedef void* (*sv_device_alloc_fn)(size_t bytes, int device, void* ctx);
typedef void (*sv_device_free_fn)(void* ptr, int device, void* ctx);

typedef struct sv_config {
    int32_t dtype;                /* SV_C64 (default) or SV_C128 */
    int32_t mode;                 /* SV_COMPRESSED (default) or SV_UNCOMPRESSED */
    uint64_t init_index;          /* initial basis state |init_index> (default 0) */
    int32_t max_group_qubits;     /* high qubits staged together per pass, g_max: 2..8, or 0
                                     (default) = automatic: the largest g <= 8 that leaves at
                                     least 4 chunk groups per pass (when n - chunk_qubits >= 4)
                                     and whose staging buffers fit in 40% of the free device
                                     memory; capped at n - chunk_qubits */
    int32_t tile_qubits;          /* qubits of one on-chip tile (0 = default for dtype) */
    int32_t pipeline_slots;       /* chunk-group buffers in flight, 2..4 (default 3) */
    int32_t renormalize;          /* 1: scale by 1/||psi|| at the next decode (default 0) */
    int32_t device;               /* CUDA device ordinal (default 0) */
    int32_t profile;              /* 1: time every decode / apply / encode launch with CUDA
                                     events on the compute stream (sv_stats t_*_s); default 0 */
    int32_t fuse_codec;           /* 1 (default): decode inside the first tile sub-pass and
                                     encode inside the last when their tiles hold whole codec
                                     blocks; 0: separate decode / encode kernels */
    int32_t jit;                  /* 1 (default): every sub-pass on 2^12-amplitude tiles runs a kernel
                                     generated for its gate sequence and compiled at run time with
                                     NVRTC (cached per process, keyed by structure, not angles);
                                     0: the table-driven phase kernel. Compilation errors fail the
                                     call with SV_ERR_CUDA. */
    int32_t relative_bound;       /* 0 (default): abs_error_bound bounds |x - xhat| for every stored
                                     component; 1: relative bound, a chunk whose largest component
                                     magnitude is m is stored with the step 2^k, k = floor(log2(2 eb m))
                                     clamped to [-60, 0], so |x - xhat| <= max(eb m, 2^-61) (spread
                                     states keep their amplitudes instead of quantising to zero).
                                     Needs eb >= 2^-23 (complex64) / 2^-29 (complex128), else
                                     SV_ERR_RANGE; the codec then runs in separate kernels (the
                                     chunk maximum precedes the encode) */
    int32_t remap_qubits;         /* 0 (default): qubits keep their positions (SWAP gates relabel
                                     them for free); 1: sv_apply_circuit may also move qubits
                                     between high (chunk-index) and low positions with physical
                                     SWAPs appended to a pass, when that runs the circuit in fewer
                                     passes (furthest-next-use rule, sv_plan_remap); logical
                                     results are unchanged. sv_grad never remaps. A remapped
                                     call leaves qubits on new positions, so repeating the same
                                     circuit runs (and, with jit, compiles) other kernels: best
                                     for one long circuit per call. */
    int32_t checkpoint_passes;    /* compressed sv_grad only. 0 (default): the reverse sweep
                                     uncomputes psi through the passes (every pass re-encodes it,
                                     so its error grows over forward and reverse passes); K > 0:
                                     the forward sweep keeps a copy of the compressed psi after
                                     every K-th pass (pageable host memory, one compressed state
                                     per checkpoint, sv_stats_t.checkpoint_bytes) and the reverse
                                     sweep resumes from it at that pass boundary */
    int32_t lambda_cache;         /* compressed sv_grad only, how lambda = H psi gets each output
                                     chunk's source chunks. 1 (default): psi decoded once into device
                                     memory when 2^n amplitudes fit in half the free device memory (or
                                     the device_alloc callback grants them), else as 2; 2: a device copy
                                     of the compressed psi (when it fits), decoded per source, so psi
                                     crosses the host link once; 0: copied from the host store per
                                     output chunk. The results are the same bit for bit. Other values:
                                     SV_ERR_ARG */
    sv_device_alloc_fn device_alloc; /* NULL (default): cudaMalloc / cudaFree. Otherwise every device
                                     allocation of the handle (state, staging, per-call scratch)
                                     goes through device_alloc / device_free (both must be set) */
    sv_device_free_fn device_free;
    void* alloc_ctx;              /* passed to device_alloc / device_free */
    void* stream;                 /* cudaStream_t of the caller, or NULL. When set, every call on the
                                     handle first waits (on the GPU) for the work the caller queued
                                     on it before the call, and the caller's stream then waits for
                                     the call's GPU work; the library's own streams do the work */
    uint64_t host_budget_bytes;   /* cap on the pinned host memory of the compressed chunk stores
                                     (sv_stats_t.host_pinned_bytes), 0 = no cap; a call that needs
                                     more fails with SV_ERR_HOST_OOM */
    double timeout_s;             /* limit of every host wait on GPU work (default 600) */
} sv_config;

typedef struct sv_stats_t {
    uint64_t passes;              /* chunk passes run since sv_create (streaming sweeps) */
    uint64_t subpasses;           /* on-chip tile sweeps over staged chunk groups */
    uint64_t groups;              /* chunk groups processed */
    uint64_t kernel_launches;     /* kernels launched by this library on this handle */
    uint64_t bytes_h2d;           /* bytes copied host -> device */
    uint64_t bytes_d2h;           /* bytes copied device -> host */
    uint64_t compressed_bytes;    /* current size of the stored state (all chunk streams) */
    uint64_t raw_bytes;           /* 2^n * sizeof(amplitude) */
    uint64_t amp_gate_updates;    /* sum over applied gates of 2^n */
    uint64_t gates_applied;
    double norm2;                 /* FP64 ||psi||^2 of the stored state after the last pass */
    double last_call_seconds;     /* wall time of the last sv_apply_circuit / sv_grad */
    double quant_step;            /* Delta of the codec (0 when uncompressed) */
    int32_t chunk_qubits;
    int32_t group_qubits;         /* g_max in use */
    /* with sv_config.profile: summed CUDA-event durations of the kernels, their
       launch counts, and their algorithmic HBM bytes (what each launch must read
       and write at least: compressed streams, amplitudes) */
    double t_decode_s, t_apply_s, t_encode_s;
    uint64_t n_decode, n_apply, n_encode;
    uint64_t alg_bytes_decode, alg_bytes_apply, alg_bytes_encode;
    /* run-time generated sub-pass kernels: compiled by this handle's calls, their
       launches, and the wall time spent generating, compiling and loading them */
    uint64_t jit_kernels_compiled, jit_launches;
    double t_jit_compile_s;
    /* with sv_config.profile: CUDA-event durations of the chunk-group copies
       (host -> device, device -> host) and of the kernels that complete fused
       encodes (offset scan, compaction) */
    double t_h2d_s, t_d2h_s, t_encode_finish_s;
    /* host wall time planning passes and looking up / compiling their kernels,
       and blocked waiting for GPU work (always collected) */
    double t_host_prepare_s, t_host_wait_s;
    /* physical SWAPs added by sv_config.remap_qubits */
    uint64_t remap_swaps;
    /* launches of generated two-vector (psi, lambda) kernels by the reverse
       sweep of sv_grad (included in jit_launches) */
    uint64_t jit_adjoint_launches;
    /* pinned host memory held by the compressed chunk stores (the state's and,
       after a compressed sv_grad, lambda's): one slot per chunk, rewritten in
       place while a chunk's new stream fits and moved to a slot with 1/32
       headroom when it grows, plus slots released by such moves */
    uint64_t host_pinned_bytes;
    /* host bytes of the psi checkpoints kept by the last compressed sv_grad
       (sv_config.checkpoint_passes), and how many there were */
    uint64_t checkpoint_bytes, checkpoints;
    /* host wall time of the last sv_grad's forward sweep, lambda = H psi, and
       reverse sweep (each ends with its GPU work complete) */
    double t_grad_forward_s, t_grad_lambda_s, t_grad_reverse_s;
} sv_stats_t;

typedef struct sv_state sv_state; /* opaque, owned by the library */

/*
 * Turn the per-launch CUDA-event timing of sv_config.profile on (1) or off (0)
 * for the following calls (the paper has no counterpart: measurement). The
 * events add a little time to every launch, so throughput is best measured
 * with it off and the breakdown taken on a separate call with it on.
 * Errors: SV_ERR_ARG for a NULL handle.
 */
int sv_set_profile(sv_state* s, int on);

/* Fill *cfg with the defaults listed above. */
void sv_config_default(sv_config* cfg);

/*
 * Create an n-qubit state |init_index> split into chunks of 2^chunk_qubits
 * amplitudes (Sec. 2, "Offline stage": partition the state vector into
 * chunks compressed independently and stored in CPU memory).
 *   n:               1..40 qubits.
 *   chunk_qubits:    8..n (compressed mode); ignored in uncompressed mode.
 *   abs_error_bound: eb > 0, pointwise bound on |x - xhat| for every real and
 *                    imaginary part stored; the codec step is the largest
 *                    power of two <= 2 eb. complex64 needs eb >= 2^-24,
 *                    complex128 eb >= 2^-30 (SV_ERR_RANGE otherwise). Ignored
 *                    in uncompressed mode.
 *   cfg:             NULL for defaults.
 *   out:             receives the handle; *out is NULL on failure.
 * Allocates pinned host memory for the compressed store and device memory
 * for the staging pipeline (or the whole state when uncompressed).
 */
int sv_create(int n, int chunk_qubits, double abs_error_bound, const sv_config* cfg, sv_state** out);

/*
 * Apply gates[0..ngates) in order (Sec. 2, "Online stage": the circuit is
 * partitioned into stages; each stage is one pass over all chunks, streamed
 * to the GPU, updated and stored back recompressed).
 *   gates:  host array; copied during the call. SWAPs relabel qubits and
 *           move no data. With sv_config.remap_qubits the call may also add
 *           physical SWAPs to its passes (sv_plan_remap lists them); logical
 *           results are the same.
 * Errors: SV_ERR_ARG (invalid gate; the state is unchanged), SV_ERR_RANGE /
 * SV_ERR_CORRUPT / SV_ERR_CUDA / SV_ERR_TIMEOUT (the state is undefined and
 * the handle should be destroyed).
 */
int sv_apply_circuit(sv_state* s, const sv_gate* gates, size_t ngates);

/*
 * *out_re = sum_j coeff_j <psi|P_j|psi> accumulated in FP64 (the
 * expectation value of a Pauli sum on the stored state; imaginary parts cancel
 * for real coefficients). Masks use logical qubits. Compressed states are
 * streamed from the host store: a sweep stages max_group_qubits high
 * (inter-chunk) qubits, decodes each chunk group and evaluates every term
 * whose high x-mask lies in the staged set; the staged sets are chosen
 * greedily to cover the terms' high x-masks (few sweeps: two for an open
 * Ising chain at n = 30, chunk_qubits = 22). Terms with more high x bits than
 * max_group_qubits, or more than 512 terms, take one sweep per distinct high
 * x-mask over chunk pairs. Errors: SV_ERR_ARG for masks beyond n qubits;
 * SV_ERR_CORRUPT / SV_ERR_CUDA / SV_ERR_TIMEOUT as sv_apply_circuit.
 */
int sv_expect(sv_state* s, const sv_pauli_term* terms, size_t nterms, double* out_re);

/*
 * Read amplitudes of logical basis indices idx[0..m) into
 * out_interleaved[2i], [2i+1] = (re, im) as FP64 (values as stored, i.e.
 * decompressed). All pointers are host memory. Indices must be < 2^n.
 */
int sv_amplitudes(sv_state* s, const uint64_t* idx, size_t m, double* out_interleaved);

/* Same as sv_amplitudes for the logical indices first .. first+count-1. */
int sv_amplitudes_range(sv_state* s, uint64_t first, size_t count, double* out_interleaved);

/*
 * The device memory of an SV_UNCOMPRESSED state, for reading on the GPU
 * between calls (the paper has no counterpart: it lets a caller use the
 * state in its own kernels without a copy, e.g. as a torch tensor).
 *   d_amps:    receives the address of 2^n interleaved complex amplitudes
 *              (complex64 or complex128 as sv_config.dtype); amplitude i is
 *              at physical index i.
 *   positions: host, NULL or n entries: the physical bit position of every
 *              logical qubit (SWAPs relabel qubits, so logical index x is at
 *              the physical index with bit positions[q] = bit q of x).
 * The memory stays owned by the handle and valid until the next call that
 * applies gates or sv_destroy; writing it is undefined.
 * Errors: SV_ERR_ARG for compressed handles or NULL arguments.
 */
int sv_device_state(sv_state* s, void** d_amps, int32_t* positions);

/*
 * *out_re + i *out_im = <a|b> = sum_x conj(a_x) b_x over logical basis
 * indices x, accumulated in FP64 on the GPU (the paper has no counterpart:
 * it measures the error the lossy store introduces, as the fidelity
 * |<ref|psi>|^2 / (||ref||^2 ||psi||^2) against a reference state).
 *   a: any handle (compressed states are streamed from the host store and
 *      decoded group by group, as sv_expect reads them; not modified).
 *   b: an SV_UNCOMPRESSED handle with the same n on the same device (its
 *      whole state is read in HBM). The two may differ in amplitude type and
 *      in their logical-to-physical qubit maps.
 * Errors: SV_ERR_ARG (b compressed, n or device differ, NULL pointers);
 * SV_ERR_CORRUPT / SV_ERR_CUDA / SV_ERR_TIMEOUT as sv_expect.
 */
int sv_inner(sv_state* a, const sv_state* b, double* out_re, double* out_im);

/*
 * Energy and gradient by the adjoint method (Jones & Gacon, arXiv
 * 2009.02823; not part of MEMQSim): resets the state to |init_index>,
 * applies the circuit with theta[param_index] as the angle of every
 * parameterised gate, forms lambda = H psi, then sweeps the circuit in
 * reverse applying U_k^dagger to psi and lambda and accumulating
 * grad[p] += Im<lambda_k|G_k|psi_k> in FP64 for every gate k with
 * param_index p (G = X, Y, Z for RX, RY, RZ).
 *   theta: host, nparams values. H: host Pauli terms. energy: host double.
 *   grad:  host, nparams doubles (overwritten), or NULL for the energy alone
 *          (the forward sweep and sv_expect: no lambda, no reverse sweep; the
 *          stored state is then psi(theta)).
 * Compressed states keep lambda as a second compressed chunk store (its
 * quantisation step is the state's times the smallest power of two >= sum
 * |coeff|, since |lambda_i| <= ||H|| <= sum |coeff|) and run
 * the reverse sweep pass by pass over both stores (re-encoding both after
 * every pass); lambda is built one chunk at a time from the source chunks
 * k ^ xh of every distinct high x-mask xh, staged 2^max_group_qubits at a
 * time (more distinct masks take several batches per chunk, accumulated on
 * the device before the chunk is encoded once).
 * On return the stored state is psi_0 as left by the reverse sweep (|init_index>
 * up to rounding and, when compressed, quantisation error); call sv_create or
 * sv_apply_circuit from a known state to continue.
 */
int sv_grad(sv_state* s, const sv_gate* gates, size_t ngates, const double* theta, size_t nparams,
            const sv_pauli_term* H, size_t nterms, double* energy, double* grad);

/*
 * The CUDA C++ sources of the sub-pass kernels sv_apply_circuit would
 * generate and compile at run time for this circuit (sv_config.jit), computed
 * on the host only (no GPU is touched). The paper has no counterpart: this
 * exposes the library's own code generator for inspection and testing.
 *   n, chunk_qubits: as in sv_create (chunk_qubits ignored when cfg->mode is
 *                    SV_UNCOMPRESSED).
 *   cfg:             NULL for defaults; dtype, mode, max_group_qubits (0 is
 *                    taken as 4 here: no device is queried), tile_qubits,
 *                    fuse_codec and remap_qubits are used.
 *   gates, ngates:   host gate list, validated as in sv_apply_circuit
 *                    (sv_grad when adjoint is set).
 *   adjoint:         0: the kernels of sv_apply_circuit; 1: those of the
 *                    reverse sweep of sv_grad (psi and lambda together, with
 *                    the gradient partials).
 *   buf, cap:        host buffer receiving the sources, each terminated by a
 *                    NUL byte, in launch order; NULL to query the size only.
 *   needed:          receives the bytes required; nkernels the number of
 *                    kernels (a sub-pass that cannot be specialised yields an
 *                    empty source and runs the table-driven kernel).
 * Errors: SV_ERR_ARG for invalid sizes or gates, or cap < *needed.
 */
int sv_jit_sources(int n, int chunk_qubits, const sv_config* cfg, const sv_gate* gates, size_t ngates, int adjoint,
                   char* buf, size_t cap, size_t* needed, size_t* nkernels);

/*
 * The chunk passes sv_apply_circuit would run, computed on the host only (no
 * GPU is touched). The paper partitions the circuit into stages but gives no
 * algorithm (Sec. 2, "Offline stage" / "Online stage"); a pass here holds the
 * gates whose non-diagonal targets lie in the chunk_qubits low qubits plus at
 * most max_group_qubits staged high qubits, and gates move ahead only past
 * gates on disjoint qubits.
 *   gates, ngates:  host gate list (validated as in sv_apply_circuit; SWAPs
 *                   relabel qubits and do not appear in the order).
 *   order:          host, >= ngates slots: indices of the executed gates in
 *                   execution order.
 *   pass_of:        host, >= ngates slots: pass of each entry of order.
 *   staged:         host, >= ngates slots: bit mask of the physical high
 *                   qubits staged by each pass.
 *   out_executed, out_passes, out_subpasses: host, counts (sub-passes are the
 *                   on-chip tile sweeps after fusion, tile_qubits 0 = default).
 * Errors: SV_ERR_ARG for invalid sizes or gates.
 */
int sv_plan(int n, int chunk_qubits, int max_group_qubits, int tile_qubits, const sv_gate* gates,
            size_t ngates, int32_t* order, int32_t* pass_of, uint64_t* staged, size_t* out_executed,
            size_t* out_passes, size_t* out_subpasses);

/*
 * sv_plan for a state with sv_config.remap_qubits = 1: the passes
 * sv_apply_circuit would run with qubit remapping. The partitioning into
 * stages is the paper's (Sec. 2, "Offline stage"); moving qubits between
 * stages is not in the paper. At the end of each pass, while a staged high
 * position holds a qubit that the remaining gates mix before the qubit of
 * some low position, the two exchange (a physical SWAP in that pass: the
 * low positions keep the qubits needed soonest), and the later gates run on
 * the new positions. The remapped plan is used only when it has fewer passes
 * than sv_plan's (*out_swaps = 0 and sv_plan's plan otherwise).
 *   order, pass_of: as in sv_plan, over the caller's gates only (the added
 *                   SWAPs are counted in *out_swaps, not listed).
 *   staged:         host, >= ngates slots: physical high positions staged by
 *                   each pass.
 *   out_swaps:      host: physical SWAPs added.
 *   swaps:          host, NULL or >= 24 * ngates slots (a pass adds at most
 *                   8 SWAPs): (pass, low position, high position) of each
 *                   added SWAP in execution order; it runs after the listed
 *                   gates of its pass, and every later gate runs on the
 *                   positions it leaves. Positions start as in sv_plan:
 *                   qubit q at q, relabelled by the caller's own SWAPs.
 *   qubits:         host, NULL or >= 4 * ngates slots: for entry k of order,
 *                   the positions its gate runs on (targets[0], targets[1],
 *                   controls[0], controls[1]; -1 where the gate has none).
 *   positions:      host, NULL or >= n slots: the position of every caller
 *                   qubit after the circuit (the logical-to-physical map the
 *                   state keeps).
 * Errors: as sv_plan.
 */
int sv_plan_remap(int n, int chunk_qubits, int max_group_qubits, int tile_qubits, const sv_gate* gates,
                  size_t ngates, int32_t* order, int32_t* pass_of, uint64_t* staged, size_t* out_executed,
                  size_t* out_passes, size_t* out_subpasses, size_t* out_swaps, int32_t* swaps, int32_t* qubits,
                  int32_t* positions);

/*
 * Copy the compressed stream of chunk k (physical chunk index, 0 <=
 * k < 2^(n - chunk_qubits)) of the stored state into h_buf (host, cap bytes);
 * *h_nbytes receives its length (also when cap is too small, which returns
 * SV_ERR_ARG). The stream is in the format of sv_codec_* (Sec. 2 "Offline
 * stage": chunks stored compressed in CPU memory). SV_ERR_ARG in uncompressed
 * mode. Physical chunk bits are logical qubits only while no SWAP has been
 * applied.
 */
int sv_chunk_stream(const sv_state* s, uint64_t k, void* h_buf, size_t cap, size_t* h_nbytes);

/* Counters and sizes of the handle. */
int sv_stats(const sv_state* s, sv_stats_t* out);

/* Human-readable description of the last error on s (never NULL; "" if none).
 * With s == NULL, the last error of a failed sv_create on this thread. */
const char* sv_last_error(const sv_state* s);

/* Release all host and device memory of s. NULL is accepted. */
void sv_destroy(sv_state* s);

/* --------------------------------------------------------------- the codec
 * Chunk codec used by the store (the paper names no compressor; Sec. 2
 * claims a state-of-the-art one). Stream format, little-endian:
 *   0  u32 magic 0x31435653 ("SVC1")     4  u16 version = 1
 *   6  u8 dtype (1 c64, 2 c128)          7  u8 c
 *   8  i32 k (step Delta = 2^k)          12 u32 nblocks = 2 * 2^c / 256
 *   16 u32 total_words                   20..31 zero
 *   32 u8 width[nblocks], i32 anchor[nblocks], u32 offset[nblocks+1], each
 *      section padded to 16 bytes; then u32 payload[total_words].
 * Blocks 0..nblocks/2-1 hold the real parts of amplitudes 256b..256b+255,
 * the rest the imaginary parts. Per block: q_j = rint(x_j / Delta) (ties to
 * even), anchor = q_0, r_0 = 0, r_j = q_j - q_{j-1}, zigzag z = 2r (r >= 0)
 * or -2r-1, width = bit length of max z, value j in bits [j w, j w + w) of
 * the block's 8 w words, offset[b+1] = offset[b] + 8 w_b.
 */

/* Largest stream size for a chunk of 2^chunk_qubits amplitudes (0 if out of range). */
size_t sv_codec_max_bytes(int chunk_qubits);

/*
 * Encode one chunk on the GPU.
 *   dtype: SV_C64 / SV_C128. chunk_qubits: 8..30. eb: as in sv_create.
 *   d_amps:   device, 2^chunk_qubits interleaved complex amplitudes.
 *   d_stream: device, capacity cap bytes (>= sv_codec_max_bytes for safety;
 *             SV_ERR_ARG if the stream would not fit).
 *   h_nbytes: host, receives the stream length.
 * Allocates and frees device scratch (packed-block staging) on every call.
 * Errors: SV_ERR_RANGE (a value outside the quantiser's range or not finite).
 */
int sv_codec_encode(int dtype, int chunk_qubits, double eb, const void* d_amps, void* d_stream,
                    size_t cap, size_t* h_nbytes);

/*
 * sv_codec_encode without any device allocation (the paper has no
 * counterpart; this is a convenience of this library).
 *
 * Who needs it: code that must not allocate GPU memory while it runs -- for
 * example a process whose device memory is already carved up by another
 * allocator (so a raw cudaMalloc would fail or fragment it), or a
 * latency-sensitive loop that cannot afford the device-wide synchronisation
 * that cudaMalloc / cudaFree imply. sv_codec_encode allocates and frees its
 * staging buffers on every call; this variant uses one staging area that is
 * part of the library image instead.
 *
 * Limits and behaviour:
 *   - chunk_qubits must be 8..SV_NOALLOC_MAX_CHUNK_QUBITS (20); larger chunks
 *     return SV_ERR_ARG. The staging area is a file-scope device array of
 *     8 MiB + 32 KiB + 256 bytes that every GPU which loads the library keeps
 *     until the process exits.
 *   - cap must be >= sv_codec_max_bytes(chunk_qubits) (SV_ERR_ARG otherwise):
 *     the stream is written in place, with no temporary.
 *   - The first call on a device looks up the staging area's device address
 *     for that device (once per device, with that device made current); make
 *     that first call before any stream capture on that device. The address
 *     is kept for the life of the process: after cudaDeviceReset (or any
 *     other teardown of the device's primary context) the library image is
 *     reloaded at a new address and later calls on that device are invalid.
 *   - All calls share the one staging area, which keeps the last call's
 *     contents. Calls are synchronous, so calls from one thread never
 *     overlap; calls from several host threads that overlap on the GPU race
 *     on the staging area and must be serialised by the caller.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 * Arguments, output and errors are those of sv_codec_encode; the stream is
 * byte-identical to sv_codec_encode's.
 */
#define SV_NOALLOC_MAX_CHUNK_QUBITS 20
int sv_codec_encode_noalloc(int dtype, int chunk_qubits, double eb, const void* d_amps, void* d_stream,
                            size_t cap, size_t* h_nbytes);

/* ----------------------------------------------------------- transfers */
/* The host <-> device copy strategies of Sec. 2 "Online stage" step (2) and
 * Table 1, timed on a 2^n-amplitude state: SV_COPY_SYNC, one bulk copy;
 * SV_COPY_ASYNC, one asynchronous copy per amplitude straight to its device
 * position (timed on the first `sample` amplitudes, 0 = all, and scaled to
 * 2^n); SV_COPY_BUFFER, one bulk copy into a device staging buffer and a
 * kernel that moves every amplitude to its position (for SV_COPY_D2H the
 * kernel gathers first). ASYNC and BUFFER place host amplitude i at device
 * index i with its low n/2 and high n - n/2 index bits exchanged; SYNC keeps
 * the order (the least time the bytes take).
 *   n: 1..34; dtype: SV_C64 / SV_C128; direction: SV_COPY_H2D / SV_COPY_D2H.
 *   seconds (host): wall time of the copies (host clock, synchronised).
 *   verified (host, may be NULL): 1 if every moved amplitude arrived at its
 *            position, 0 otherwise.
 * Allocates (and frees) 2^n amplitudes of pinned host memory and one or two
 * device arrays of that size. Errors: SV_ERR_ARG, SV_ERR_HOST_OOM,
 * SV_ERR_DEVICE_OOM, SV_ERR_CUDA. */
#define SV_COPY_SYNC 0
#define SV_COPY_ASYNC 1
#define SV_COPY_BUFFER 2
#define SV_COPY_H2D 0
#define SV_COPY_D2H 1
int sv_copy_probe(int n, int dtype, int strategy, int direction, uint64_t sample, double* seconds, int* verified);

/* sv_codec_encode with the relative bound of sv_config.relative_bound: the
 * chunk's step follows its largest component magnitude m (k in the stream
 * header), |x - xhat| <= max(eb m, 2^-61). eb >= 2^-23 (complex64) / 2^-29
 * (complex128), else SV_ERR_RANGE; otherwise as sv_codec_encode. The stream
 * decodes with sv_codec_decode. */
int sv_codec_encode_relative(int dtype, int chunk_qubits, double eb, const void* d_amps, void* d_stream,
                             size_t cap, size_t* nbytes);

/*
 * Decode one chunk stream of nbytes bytes (device) into d_amps (device,
 * 2^chunk_qubits interleaved complex). SV_ERR_CORRUPT if the stream fails
 * validation (magic, sizes, widths <= 32, offsets consistent with widths).
 */
int sv_codec_decode(int dtype, int chunk_qubits, const void* d_stream, size_t nbytes, void* d_amps);

#ifdef __cplusplus
}
#endif
#endif /* SV_GB300_SV_H */
