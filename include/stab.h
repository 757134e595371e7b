/*
 * stab.h -- C interface of the GB300 Pauli-coefficient propagation library.
 *
 * The library implements the propagation stage ("Map", Sec. IV-B) of the
 * extended stabilizer formalism of arXiv 2502.10685: every stabilizer
 * generator Z_k of |0^n> (Eq. (1)) and every observable is held as a dense
 * FP64 vector of its 4^n Pauli-string coefficients, and each gate of a
 * parameterized circuit maps that vector to the coefficients of g P g^dagger
 * (Sec. II-A: Clifford gates map strings to signed strings; R_x, R_y, R_z mix
 * strings by cos/sin as in Table I).  Observables are propagated backward
 * (U^dagger O U) and <0^n| O |0^n> is read from the strings made of I and Z.
 *
 * Conventions (all entry points):
 *  - Every function returns a status: STAB_OK (0) or a negative STAB_E_* code.
 *    No C++ exception crosses this interface.  On an error the context keeps
 *    the state it had before the call.
 *  - Input arrays are owned by the caller and are copied or consumed before the
 *    call returns, unless a parameter says it is a device pointer that must
 *    stay valid until the next synchronizing call.
 *  - Work is queued on the context's stream(s); results written to host
 *    memory are complete when the call returns, results written to device
 *    memory are complete after stab_synchronize() or an event on the stream.
 *  - A context is used by one host thread at a time.
 *
 * Coefficient layout on the device and in every generator output:
 *    index(P) = z | (x << n),  bit q of x (z) set iff the letter on qubit q is
 *    X or Y (Z or Y);  I = (0,0), X = (1,0), Z = (0,1), Y = (1,1).
 * The strings made of I and Z (x = 0) are the contiguous block [0, 2^n).
 */
#ifndef STAB_LIB_INTERFACE_H
#define STAB_LIB_INTERFACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STAB_VERSION 1

/* ---------------------------------------------------------------- status */
#define STAB_OK 0
#define STAB_E_INVAL (-1)     /* null pointer, unknown opcode, qubit >= n, q0 == q1, bad term */
#define STAB_E_RANGE (-2)     /* n outside [1, STAB_MAX_QUBITS], slot outside [0, n_params), size */
#define STAB_E_NOMEM (-3)     /* device allocation failed, or a request does not fit */
#define STAB_E_TIMEOUT (-4)   /* a bounded device wait gave up (status read back on the host) */
#define STAB_E_NONFINITE (-5) /* an angle or coefficient is NaN or infinite */
#define STAB_E_CUDA (-6)      /* CUDA runtime error; stab_last_cuda_error() returns its code */
#define STAB_E_STATE (-7)     /* call out of order (e.g. expectation before a circuit is loaded) */
#define STAB_E_BUSY (-8)      /* server queue full */

#define STAB_MAX_QUBITS 12

/* ---------------------------------------------------------------- gates */
/* Opcodes.  H, S and the rotations are Table I; CX is map_CX of Sec. III-C
 * (q0 = control, q1 = target).  S^dagger, X, Y, Z and CZ are the standard
 * Clifford gates; each is a composition of the paper's rules.  Rotations are
 * R_s(theta) = exp(-i theta s / 2), the convention under which Table I and
 * Example 1 hold. */
enum stab_op {
    STAB_H = 0, STAB_S = 1, STAB_SDG = 2, STAB_X = 3, STAB_Y = 4, STAB_Z = 5,
    STAB_CX = 6, STAB_CZ = 7, STAB_RX = 8, STAB_RY = 9, STAB_RZ = 10
};

/* One instruction {g, w, theta} of Sec. III-A.  8 bytes.
 *  op     stab_op
 *  q0     wire (control of CX, first qubit of CZ)
 *  q1     second wire of CX / CZ, else ignored
 *  flags  reserved, must be 0
 *  param  rotations: index of the angle in the thetas array (several gates may
 *         share a slot; gradients sum over them); other gates: ignored (-1). */
typedef struct stab_gate {
    uint8_t op, q0, q1, flags;
    int32_t param;
} stab_gate;

/* One observable term coeff * P(x, z); bit q of x / z as in the layout above. */
typedef struct stab_term {
    double coeff;
    uint64_t x, z;
} stab_term;

/* ---------------------------------------------------------------- options */
enum stab_kernel {
    /* The library's choice.  n <= 6: vectors resident in shared memory; plans of
     * 64 or more passes are cut in two and both parts run at once (the
     * generators at n <= 4 through the second part's transfer matrix, <O> and
     * gradients meeting at the cut).  n >= 7: vectors in HBM, passes grouped
     * into shared-memory tiles where the vectors are small, else one fused pass
     * per launch (gradients again meet at the cut).  Batches pick their CTAs
     * per SM by timing a sample of their units. */
    STAB_KERNEL_AUTO = 0,
    STAB_KERNEL_RESIDENT = 1,  /* n <= 6: one CTA per vector through the whole circuit, never cut */
    STAB_KERNEL_STREAMED = 2,  /* vector in HBM, fused passes (any n) */
    STAB_KERNEL_PLAIN = 3      /* the comparison form: one pass per gate, no fusion, no cut; one
                                  resident launch per circuit at n <= 6, one launch per gate above */
};

/* Device allocator hooks.  With alloc == NULL the library uses cudaMallocAsync
 * / cudaFreeAsync on its stream.  The Python binding passes PyTorch's caching
 * allocator here. */
typedef void *(*stab_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*stab_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct stab_opts {
    int32_t device;        /* CUDA device ordinal, -1 = the current device */
    int32_t kernel;        /* stab_kernel */
    int32_t fuse;          /* 1 (default): group per-wire runs and CX runs (Sec. III-A) */
    int32_t stream_given;  /* 1: queue on `stream` even when it is NULL (the legacy default
                              stream); 0: on `stream` if non-NULL, else on a stream the
                              context creates */
    void *stream;          /* cudaStream_t */
    stab_alloc_fn alloc;
    stab_free_fn free;
    void *alloc_user;
} stab_opts;

/* Fills *opts with the defaults (device -1, AUTO, fuse 1, own stream, cudaMallocAsync). */
void stab_default_opts(stab_opts *opts);

/* ---------------------------------------------------------------- context */
typedef struct stab_ctx stab_ctx;

/* Creates a context for n qubits (1 <= n <= STAB_MAX_QUBITS).  opts may be
 * NULL.  The context owns the device vectors: n generators of 4^n doubles and
 * the work vectors of expectation and gradient calls.  The first AUTO context
 * of each n in the process may run the path tuner (stab_path_tune) on the
 * device, on streams of its own, allocating through opts' hooks; it
 * synchronizes, so do not create contexts while work on the device must not
 * be waited for (for instance during a global-mode stream capture).
 * Errors: STAB_E_RANGE (n), STAB_E_INVAL (out NULL), STAB_E_CUDA, STAB_E_NOMEM. */
int stab_create(int n, const stab_opts *opts, stab_ctx **out);

/* Releases every device buffer and stream the context owns.  NULL is a no-op. */
int stab_destroy(stab_ctx *ctx);

/* Loads a circuit (Sec. III-A dividing + encoding): validates the m gate
 * records (host memory), plans the fused passes, uploads them and encodes the
 * n_params angles (host memory).  Replaces any previous circuit.  m = 0 is the
 * identity circuit.  Errors: STAB_E_INVAL (bad opcode, qubit, q0 == q1),
 * STAB_E_RANGE (param slot), STAB_E_NONFINITE (angle), STAB_E_CUDA. */
int stab_load_circuit(stab_ctx *ctx, const stab_gate *gates, int64_t m, const double *thetas,
                      int64_t n_params);

/* Replaces the angles of the loaded circuit.  thetas has the loaded n_params
 * entries, in host memory (is_device = 0) or device memory (is_device = 1,
 * read on the context stream).  Errors: STAB_E_STATE (no circuit),
 * STAB_E_NONFINITE (host angles only), STAB_E_CUDA. */
int stab_set_params(stab_ctx *ctx, const double *thetas, int is_device);

/* Evolves the n generators of |0^n> (Eq. (1)) through the loaded circuit:
 * generator k becomes U Z_k U^dagger.  Asynchronous.  Errors: STAB_E_STATE. */
int stab_run_generators(stab_ctx *ctx);

/* stab_load_circuit followed by stab_run_generators. */
int stab_apply_circuit(stab_ctx *ctx, const stab_gate *gates, int64_t m, const double *thetas,
                       int64_t n_params);

/* Copies the n evolved generators, n x 4^n doubles in the layout above, to
 * out (host memory if out_is_device == 0, then synchronizing; device memory
 * otherwise, queued on the context stream).  Errors: STAB_E_STATE (never run). */
int stab_get_generators(stab_ctx *ctx, double *out, int out_is_device);

/* Device pointer of the generator block (n x 4^n doubles), valid until the
 * next load/run call or stab_destroy.  NULL before the first run. */
const double *stab_generators_device(stab_ctx *ctx);

/* <0^n| U^dagger O U |0^n> for O = sum of n_terms terms (host memory) and the
 * loaded circuit U: O is propagated backward through the circuit and the
 * coefficients of the strings made of I and Z are summed (fixed-order tree).
 * *out (host) is written before return.  Errors: STAB_E_INVAL (x or z has a
 * bit >= n), STAB_E_NONFINITE, STAB_E_STATE. */
int stab_expect(stab_ctx *ctx, const stab_term *O, int64_t n_terms, double *out);

/* Uploads an observable O = sum of n_terms terms (host memory) for the
 * asynchronous calls below; equal strings are merged.  Errors: STAB_E_INVAL
 * (x or z has a bit >= n), STAB_E_NONFINITE. */
int stab_set_observable(stab_ctx *ctx, const stab_term *O, int64_t n_terms);

/* <O> of the loaded observable and circuit, written to out_dev (device
 * memory, one double).  Queued on an internal stream that the context stream
 * then waits for, so work queued later on the context stream sees the value.
 * Errors: STAB_E_STATE (no circuit or no observable). */
int stab_expect_async(stab_ctx *ctx, double *out_dev);

/* Adjoint gradient of the loaded observable: expect_dev (device, may be NULL)
 * receives <O>, grads_dev (device) n_params doubles.  Queued like
 * stab_expect_async.  At n <= 4 (AUTO kernel, long circuits) the gradient is
 * cut into the parts of the generators' split sweep and takes its vectors at
 * the cuts from that sweep: when none was made for the current angles it is
 * queued first on the context stream (as by stab_run_generators, whose
 * results it leaves valid for reuse), then the gradient on the internal
 * stream.  Same for stab_expect_async in that form. */
int stab_grad_async(stab_ctx *ctx, double *expect_dev, double *grads_dev);

/* How the last gradient's plan is cut: *parts receives K >= 2 when it is cut
 * into the K parts of the generators' split sweep (n <= 4; the pairs at the
 * cuts come from that sweep), 1 when it uses the meet-in-the-middle or a
 * streamed sweep, 0 before any gradient since the circuit was loaded.
 * Errors: STAB_E_INVAL (ctx or parts NULL). */
int stab_grad_parts(stab_ctx *ctx, int32_t *parts);

/* Gradient of <O> with respect to every angle slot, by one adjoint reverse
 * sweep.  expect_out (may be NULL) receives <O>; grads_out receives n_params
 * doubles (host memory).  Errors as stab_expect. */
int stab_grad(stab_ctx *ctx, const stab_term *O, int64_t n_terms, double *expect_out,
              double *grads_out);

/* <0^n| U^dagger O U |0^n> without any device allocation, for callers that
 * must not allocate device memory (a program that reserves its device budget
 * at start-up and allows no growth later, or code running inside a framework
 * whose allocator owns the device).  The paper has no counterpart: this is a
 * deployment entry point around the same propagation as stab_expect with
 * STAB_KERNEL_STREAMED.
 *  n, gates (m records), thetas (n_params), O (n_terms terms): host memory,
 *    meaning as in stab_load_circuit and stab_expect; out: host double.
 *  stream: cudaStream_t to queue on (NULL = the legacy default stream of
 *    the current device); it must belong to the current device
 *    (STAB_E_INVAL otherwise).  The call waits for its own work before
 *    returning.
 * Everything the call needs on the device -- the planned passes, the angles,
 * the terms and two working vectors of 4^n doubles -- lives in one 16 MiB
 * workspace that the library holds as a static device array on every GPU
 * that loads it, until the process exits.  A problem that does not fit
 * (roughly n <= 9 for short circuits; fewer qubits for very long ones)
 * returns STAB_E_RANGE.  The first call on a device looks up the workspace's
 * device address with that device current and keeps it for the life of the
 * process, so the call is not supported after cudaDeviceReset() of a device
 * it has run on.  Every call copies from host memory and synchronizes its
 * stream, so it must not be called while its stream (or, in global capture
 * mode, any stream) is being captured.  All calls share the workspace: calls
 * whose work overlaps on the GPU (other threads, other streams) race and give
 * wrong results, so serialize them.  Errors: as stab_load_circuit and
 * stab_expect, STAB_E_RANGE (too large), STAB_E_INVAL (stream of another
 * device), STAB_E_CUDA. */
int stab_expect_static(int n, const stab_gate *gates, int64_t m, const double *thetas,
                       int64_t n_params, const stab_term *O, int64_t n_terms, double *out,
                       void *stream);

/* ---------------------------------------------------------------- batches */
/* Many independent circuits of different sizes evaluated by one persistent
 * launch (replayed from a CUDA graph): every generator of a generator item
 * and the observable of an expectation item is one unit of work; CTAs take
 * units longest first.  The 2m parameter-shift copies of a circuit (Sec. I)
 * are expectation items that differ only in their angles. */
#define STAB_BATCH_MAX_QUBITS 8

enum stab_item_kind { STAB_ITEM_GENERATORS = 0, STAB_ITEM_EXPECT = 1 };

typedef struct stab_batch_item {
    int32_t n;               /* qubits, 1 <= n <= STAB_BATCH_MAX_QUBITS */
    int32_t kind;            /* stab_item_kind */
    const stab_gate *gates;  /* m records, host memory, rules of stab_load_circuit */
    int64_t m;
    const double *thetas;    /* n_params angles, host memory */
    int64_t n_params;
    const stab_term *obs;    /* STAB_ITEM_EXPECT: n_terms terms, host memory */
    int64_t n_terms;
} stab_batch_item;

typedef struct stab_batch stab_batch;

/* Validates, plans and uploads count items (all host arrays are copied before
 * return).  opts may be NULL.  opts->kernel sets the residency: AUTO times
 * candidate launches on a sample of the units (prefixes of their streams) and
 * picks which vectors stay in shared memory (n <= 4, 5 or 6; larger ones in a
 * per-CTA global slab) and how many CTAs run per SM; RESIDENT keeps every
 * n <= 6 vector in shared memory; STREAMED keeps n <= 4 there and the rest in
 * slabs (both at the largest residency).  Errors: as stab_load_circuit /
 * stab_expect, STAB_E_RANGE (n > 8 or count < 1), STAB_E_NOMEM, STAB_E_CUDA. */
int stab_batch_create(const stab_batch_item *items, int64_t count, const stab_opts *opts,
                      stab_batch **out);

/* Queues one evaluation of every item (asynchronous). */
int stab_batch_run(stab_batch *b);

/* The same call under the name of the batch step of the propagation path
 * (all items of a created batch, parameter-shift copies included, in one
 * persistent launch). */
int stab_apply_batch(stab_batch *b);

/* After stab_batch_run: <O> of every item into out[0 .. count) (host; NaN for
 * generator items).  Synchronizes.  Errors: STAB_E_STATE (never run),
 * STAB_E_TIMEOUT. */
int stab_batch_expectations(stab_batch *b, double *out);

/* After stab_batch_run: the n x 4^n generators of generator item `item`
 * (host memory if out_is_device == 0, synchronizing; else device memory). */
int stab_batch_generators(stab_batch *b, int64_t item, double *out, int out_is_device);

/* units: vectors in the batch; grid: CTAs of the persistent launch;
 * ctas_per_sm and smem_max_n: the chosen residency (vectors of up to
 * smem_max_n qubits in shared memory, larger ones in a per-CTA global slab;
 * with STAB_KERNEL_AUTO both are picked by timing candidates at creation).
 * Any pointer may be NULL. */
int stab_batch_info(stab_batch *b, int64_t *units, int32_t *grid, int32_t *ctas_per_sm,
                    int32_t *smem_max_n);

int stab_batch_destroy(stab_batch *b);

/* ---------------------------------------------------------------- serving */
/* A request server with continuous batching: requests (an expectation value
 * or an adjoint gradient of one circuit) are queued as they arrive and
 * admitted whenever a slot and enough HBM budget are free; requests join
 * while others are running and leave as soon as they finish.  The paper has
 * no counterpart (it evaluates one circuit per call).  Two engines run the
 * admitted requests:
 *  - STAB_SERVE_ITERATE (default): requests of n <= iter_max_n are advanced together
 *    by one persistent kernel launch per iteration; each launch moves every
 *    admitted request a slice of its instruction streams further (as many
 *    4 KiB chunks as take about iter_slice_us by the measured cost of its
 *    kind of unit; before a kind is measured, iter_chunks chunks at n = 4, a
 *    quarter of that per extra qubit, at least one), its vectors staying in
 *    its own device memory between launches.  New requests join at the next
 *    launch.  Larger requests run as in STAB_SERVE_CONTEXTS, beside them.
 *  - STAB_SERVE_CONTEXTS: each admitted request runs on its own pooled
 *    context and streams, so the kernels of all admitted requests overlap on
 *    the device; contexts keep their device vectors between requests.
 * Within an engine a result does not depend on the other requests or on
 * when the request was admitted (its passes run in the same order on the
 * same data whatever the slicing); the two engines use different kernels and
 * agree to rounding. */
typedef struct stab_server stab_server;

/* Admission order.  FIFO: the oldest queued request.  SHORTEST: the queued
 * request with the least estimated work (gates x 4^n, three times that for a
 * gradient), oldest first among equals -- unless the oldest queued request
 * has waited longer than aging_s, which is then admitted first, so a large
 * request waits at most about aging_s plus the time for budget to free up. */
enum stab_serve_policy { STAB_SERVE_FIFO = 0, STAB_SERVE_SHORTEST = 1 };

enum stab_serve_engine { STAB_SERVE_ITERATE = 0, STAB_SERVE_CONTEXTS = 1 };

typedef struct stab_server_opts {
    int32_t device;        /* CUDA device ordinal, -1 = current */
    int32_t max_active;    /* requests admitted at once (0 = 64) */
    int64_t hbm_budget;    /* bytes of request state admitted at once (0 = 32 GiB) */
    int32_t planners;      /* host threads that plan and launch requests (0 = 4) */
    int32_t policy;        /* stab_serve_policy: which queued request is admitted next */
    int32_t engine;        /* stab_serve_engine */
    int32_t iter_chunks;   /* ITERATE: chunks per slice at n = 4 (0 = 32) */
    int32_t iter_smem_kb;  /* ITERATE: KiB of shared memory per CTA for vectors (0 = 32, <= 200);
                              a request whose working vectors fit runs in shared memory,
                              others in their own device memory */
    int32_t iter_max_n;    /* ITERATE: largest n the iteration engine takes (0 = 6, 1 .. 8);
                              larger requests run on contexts (one CTA per vector leaves a
                              4^7 or 4^8 vector latency-bound) */
    double aging_s;        /* SHORTEST: aging bound in seconds (0 = 4 s, < 0 = none) */
    stab_alloc_fn alloc;   /* device memory of the server, its contexts and requests; NULL:
                              cudaMallocAsync / cudaFreeAsync (both NULL or both set) */
    stab_free_fn free;
    void *alloc_user;
    double iter_slice_us;  /* ITERATE: target length of one unit's slice in microseconds (0 =
                              400; < 0 = the static budget of iter_chunks only).  The launch
                              records how long every slice took; per kind of unit (n, vector or
                              pair, in shared memory or not) the engine keeps an estimate of a
                              chunk's cost and gives each unit as many chunks as fill the
                              target, so the units of one launch end together; until a kind
                              has been measured it gets the static budget. */
} stab_server_opts;

enum stab_request_kind { STAB_REQ_EXPECT = 0, STAB_REQ_GRAD = 1 };

typedef struct stab_request {
    int32_t n;               /* 1 <= n <= STAB_MAX_QUBITS */
    int32_t kind;            /* stab_request_kind */
    const stab_gate *gates;  /* host memory, copied by stab_server_submit */
    int64_t m;
    const double *thetas;
    int64_t n_params;
    const stab_term *obs;
    int64_t n_terms;
} stab_request;

typedef struct stab_result {
    int32_t status;          /* STAB_OK or this request's error */
    int32_t n_params;
    double expect;           /* <O> */
    double submit_s;         /* server clock (seconds since creation) */
    double admit_s;          /* admitted: planning and launch started */
    double done_s;           /* results on the host */
} stab_result;

/* Admission footprint of a request: max(n 4^n 8, 4^n 8 x (4 for <O>, 12 for
 * a gradient: the vectors of the split sweeps)) bytes plus 96 bytes per gate,
 * plus at n <= 4 the split sweep's transfer matrices (8 x 16^n bytes each: two
 * at n = 4, up to min(49, 160 / (4^n - 1)) at n <= 3), its n + 1 first-part
 * vectors and the pairs at the cuts (two vectors per matrix),
 * plus, for a gradient, the adjoint's partial dot sums: per CTA of the
 * streamed sweep above n = 6, per thread of the resident sweep at n <= 5
 * (8 bytes x gates x 32, 32, 32, 64, 256 threads at n = 1..5, while that
 * stays within 256 MiB), as a bound on one per rotation. */
int64_t stab_request_footprint(const stab_request *req);

/* opts may be NULL (all defaults).  Errors: STAB_E_INVAL (unknown policy or
 * engine, iter_chunks < 0, iter_smem_kb outside [0, 200], only one of alloc /
 * free set), STAB_E_CUDA. */
int stab_server_create(const stab_server_opts *opts, stab_server **out);

/* Queues a copy of *req; *id identifies it.  Invalid requests are accepted
 * and complete with their error status.  A request whose footprint exceeds
 * the whole budget completes with STAB_E_NOMEM. */
int stab_server_submit(stab_server *s, const stab_request *req, int64_t *id);

/* Waits up to timeout_s (< 0: forever) for request id.  grads (host, may be
 * NULL) receives the n_params gradient entries of a gradient request.  A
 * successful wait hands the results out and releases the request: its id is
 * unknown afterwards.  Errors: STAB_E_INVAL (unknown id), STAB_E_TIMEOUT (not
 * done in time; the request stays queued or running). */
int stab_server_wait(stab_server *s, int64_t id, double timeout_s, stab_result *out,
                     double *grads);

/* *done = 1 when request id has completed (it stays known until waited for). */
int stab_server_poll(stab_server *s, int64_t id, int32_t *done);

/* stab_server_submit and stab_server_poll under the names of the serving
 * step of the propagation path. */
int stab_serve_submit(stab_server *s, const stab_request *req, int64_t *id);
int stab_serve_poll(stab_server *s, int64_t id, int32_t *done);

/* Counters: requests submitted, completed, admitted now, bytes admitted now. */
int stab_server_stats(stab_server *s, int64_t *submitted, int64_t *completed, int64_t *active,
                      int64_t *bytes_in_use);

/* Waits for every queued request, then releases the server. */
int stab_server_destroy(stab_server *s);

/* Density matrix rho = |psi><psi| of psi = U|0^n> for the loaded circuit (the
 * paper's decoding and toDM() step, Sec. III-D and IV-C): the coefficients of
 * 2^n |0><0| are propagated forward and decoded as rho = 2^-n sum_P r_P P.
 * out: 2^n x 2^n complex entries as interleaved (re, im) doubles, row-major,
 * 2 x 4^n doubles; row and column index bit q is qubit q.  Host memory if
 * out_is_device == 0 (synchronizing), else device memory (queued).
 * Errors: STAB_E_STATE (no circuit), STAB_E_CUDA, STAB_E_NOMEM. */
int stab_density_matrix(stab_ctx *ctx, double *out, int out_is_device);

/* Waits for all work queued by the context. */
int stab_synchronize(stab_ctx *ctx);

/* ---------------------------------------------------------------- sparse term lists */
/* The sparse representation of Sec. II-B: a stabilizer or observable held as
 * its list of terms lambda * P (the (lambda, I) pairs), whose length is the
 * stabilizer order n' of Fig. 1.  The list is propagated on the device while
 * n' stays small, so n may go up to STAB_SPARSE_MAX_QUBITS: Clifford gates map
 * each term to one signed term, a rotation gives each anticommuting term its
 * partner string (u' = c u - s v, v' = s u + c v, Table I), so n' at most
 * doubles per rotation.  Keys use the layout above (z | x << n).  Terms whose
 * coefficient is exactly zero are dropped.  The order of the list is
 * deterministic (the images of each term in input order).
 * Expectations switch to the dense path (stab_ctx) once n' exceeds a
 * threshold, for n <= STAB_MAX_QUBITS. */
#define STAB_SPARSE_MAX_QUBITS 32

typedef struct stab_sparse stab_sparse;

typedef struct stab_sparse_info {
    int64_t order_final;   /* terms in the list when the sparse path ended */
    int64_t order_max;     /* longest list seen */
    int64_t steps;         /* steps run on the list (Clifford runs + rotations) */
    int64_t dense_gates;   /* gates left to the dense path at the switch; -1: no switch */
    int32_t regrows;       /* times the list capacity was enlarged */
    int32_t reserved;
} stab_sparse_info;

/* Creates a sparse context for n qubits (1 <= n <= STAB_SPARSE_MAX_QUBITS)
 * holding up to max_terms terms (1 <= max_terms <= 2^30); the buffers start
 * small and grow by 8x when a step would overflow them (the step is then
 * re-run), up to max_terms.  Device memory is about 72 bytes per term of
 * capacity.  opts as for stab_create (kernel and fuse apply to the dense
 * path it switches to).
 * Errors: STAB_E_RANGE (n, max_terms), STAB_E_INVAL, STAB_E_CUDA, STAB_E_NOMEM. */
int stab_sparse_create(int n, int64_t max_terms, const stab_opts *opts, stab_sparse **out);
int stab_sparse_destroy(stab_sparse *s);

/* Validates and copies a gate list and its angles (host memory), as
 * stab_load_circuit.  Errors: STAB_E_INVAL, STAB_E_RANGE, STAB_E_NONFINITE. */
int stab_sparse_load_circuit(stab_sparse *s, const stab_gate *gates, int64_t m,
                             const double *thetas, int64_t n_params);

/* Order above which an expectation continues on the dense 4^n vector (the
 * rest of the circuit through the dense path); 0 = never.  Only for
 * n <= STAB_MAX_QUBITS.  Default: 4^n / 16 for n <= 12, else 0.
 * Errors: STAB_E_RANGE (negative, or nonzero with n > STAB_MAX_QUBITS). */
int stab_sparse_set_dense_threshold(stab_sparse *s, int64_t order);

/* <0^n| U^dagger O U |0^n>: O (host terms, duplicates summed) is propagated
 * backward as a list, then its x-free coefficients are summed in list order.
 * info may be NULL.  Synchronizing.
 * Errors: STAB_E_STATE (no circuit), STAB_E_INVAL (bad term), STAB_E_RANGE
 * (the list outgrew max_terms and no dense switch was possible), STAB_E_CUDA,
 * STAB_E_NOMEM. */
int stab_sparse_expect(stab_sparse *s, const stab_term *O, int64_t n_terms, double *out,
                       stab_sparse_info *info);

/* U Z_k U^dagger as a term list: writes up to max_out terms to out (host)
 * and the number of terms to *n_out; when *n_out > max_out nothing is
 * written and STAB_E_RANGE is returned.  Synchronizing.
 * Errors: STAB_E_STATE, STAB_E_RANGE (k, list size), STAB_E_CUDA, STAB_E_NOMEM. */
int stab_sparse_generator(stab_sparse *s, int k, int64_t max_out, stab_term *out,
                          int64_t *n_out, stab_sparse_info *info);

/* The order after each step of the last expect / generator call (the
 * stabilizer order curve of Fig. 1): writes min(count, max) values and sets
 * *count to the number of steps run. */
int stab_sparse_order_history(stab_sparse *s, int64_t *orders, int64_t max, int64_t *count);

/* Number of qubits, loaded gates and fused passes of the current plan. */
int stab_plan_info(stab_ctx *ctx, int64_t *n_gates, int64_t *n_passes, int32_t *kernel);

/* The cut of the split resident sweeps of the current plan (n <= 6, AUTO
 * kernel, fused).  <O> = <lambda, r> for any cut of the circuit, since every
 * gate's map is orthogonal (Sec. II): r = rho_0 through passes [0, cut) and
 * lambda = O backward through [cut, n_passes) run at once; for n <= 4 the
 * generators are T a_k, a_k = Z_k through [0, cut) and T the transfer matrix
 * of [cut, n_passes).  Writes *cut (-1: no split; the plan runs as one
 * sweep), *gen_units (vectors of the generators' split sweep -- the n
 * generators and rho_0 through [0, cut), the 4^n - 1 columns of T; 0 when not
 * split; stab_density_matrix uses the same sweep, r = T r_1) and
 * *expect_units (of the expectation's own launch, 0 when not split).  At
 * n <= 3 a long plan is cut into K >= 3 parts of equal pass counts (cut = the
 * first cut): the sweep carries the K - 1 later parts' transfer matrices,
 * the generators are T_K ... T_2 a_k, and <O> = sum_P o_P (T_K ... T_2 r_1)_P
 * reuses the sweep made for the same angles (*expect_units = 0).
 * Any output pointer may be NULL.  Errors: STAB_E_INVAL (ctx NULL). */
int stab_split_info(stab_ctx *ctx, int64_t *cut, int32_t *gen_units, int32_t *expect_units);

/* Number of kernels this context launched since creation (all entry points). */
int64_t stab_launch_count(stab_ctx *ctx);

/* Bytes the context copied host -> device and device -> host since creation. */
int stab_transfer_bytes(stab_ctx *ctx, int64_t *h2d, int64_t *d2h);

/* Human-readable name of a status code (static storage). */
const char *stab_error_string(int status);

/* CUDA error code behind the last STAB_E_CUDA returned on this thread. */
int stab_last_cuda_error(void);

int stab_version(void);

/* Self-test of failure reporting: runs one small kernel whose thread 0 waits
 * on a shared-memory barrier that nothing ever completes, giving up after
 * `polls` polls exactly as every bounded wait of the library does, and
 * returns what the host reads back: STAB_E_TIMEOUT when the bound was reached
 * (any polls > 0), STAB_OK for polls == 0.  The device stays usable.
 * Errors: STAB_E_RANGE (polls < 0), STAB_E_CUDA. */
int stab_selftest_bounded_wait(int64_t polls);

/* Self-test of the host planner (no device work): plans the m gates (host
 * memory) in plan mode `mode` (0 fused, 1 gradient, 2 one pass per gate,
 * 3 one map per wire run) both in parallel chunks and sequentially, with
 * their forward and backward instruction streams, and returns STAB_OK when
 * every array is byte-identical and the streams built as two pieces at once
 * (long streams on the host pool) apply the same pulls and passes in the same
 * order as the one-piece streams; STAB_E_STATE when any of this fails.
 * Errors: STAB_E_INVAL / STAB_E_RANGE (gates as for stab_load_circuit, mode). */
int stab_selftest_plan(int n, const stab_gate *gates, int64_t m, int64_t n_params, int mode);

/* Host-only check of the cut alignment between a circuit's generator plan
 * (one 3x3 map per wire run) and its gradient plan (every rotation its own
 * op): for every pass of the generator plan that starts a unit (a two-qubit
 * pass, or the passes of one wire run), the gradient-plan pass the aligner
 * maps it to must hold before it exactly the same rotations (by ordinal) and
 * the same number of two-qubit gates; where the aligner refuses, the two
 * plans' unit sequences must really differ.  *aligned receives how many
 * passes were aligned (0 when the aligner refused).  STAB_OK, or
 * STAB_E_STATE when a check fails.  Errors: STAB_E_INVAL / STAB_E_RANGE
 * (gates as for stab_load_circuit). */
int stab_selftest_align(int n, const stab_gate *gates, int64_t m, int64_t n_params,
                        int64_t *aligned);

/* ---------------------------------------------------------------- path tuner */
/* How a context of n qubits with the STAB_KERNEL_AUTO kernel runs, for one GPU
 * model.  The paper has no counterpart (its CPU pipeline has one form).  The
 * values are picked by timing the candidates on a probe circuit (a layered
 * ansatz: R_x, R_y, R_z on every qubit, then a CNOT ring) on the GPU the
 * first time an AUTO context of that n is created in the process, and kept
 * in a process-wide cache keyed by the GPU's name and n.  Environment:
 * STAB_PATH_TUNE=0 leaves the built-in defaults in place of tuning (entries
 * already in the cache are still used); STAB_PATH_CACHE=<file> loads the cache
 * from that file before the first lookup and writes it back after each
 * tuning. */
typedef struct stab_path_choice {
    int32_t resident;          /* n <= 6: 1 = each vector resident in shared memory on one CTA,
                                  0 = vectors streamed through HBM (grid-wide passes) */
    int32_t resident_adjoint;  /* n <= 6: 1 = gradients by the resident adjoint, 0 = streamed */
    double gen_cut;            /* n <= 4: where the generators' split sweep cuts the plan, as a
                                  fraction of its passes (0.3 .. 0.7): the end of the first part */
    int64_t tile_limit;        /* streamed plans: consecutive wire passes share one tile-fused
                                  launch while vectors x 4^n <= tile_limit, else one launch
                                  per pass (>= 0) */
    int32_t tuned;             /* 1: measured on this GPU model; 0: the built-in defaults */
    int32_t gen_parts;         /* n = 4: 2 = the plan cut once at gen_cut (the generators through
                                  one transfer matrix); 3 = a first part of gen_cut of the passes
                                  and two equal parts after it (the generators through a chain of
                                  two transfer matrices whose columns run four to an SM) */
} stab_path_choice;

/* The built-in defaults for n qubits: resident and resident_adjoint 1,
 * gen_cut 0.56 at n = 4 (0.5 below), tile_limit 2^17, tuned 0, gen_parts 2.
 * Errors: STAB_E_RANGE (n), STAB_E_INVAL (out NULL). */
int stab_path_defaults(int n, stab_path_choice *out);

/* The cached choice for (gpu_name, n).  Errors: STAB_E_STATE (no entry),
 * STAB_E_RANGE (n), STAB_E_INVAL (NULL pointer). */
int stab_path_lookup(const char *gpu_name, int n, stab_path_choice *out);

/* Stores a choice for (gpu_name, n), replacing any entry; later AUTO contexts
 * of that n on a GPU of that name use it.  gpu_name: at most 255 bytes, no
 * tab or newline.  Errors: STAB_E_INVAL (a value outside its range, a bad
 * name), STAB_E_RANGE (n). */
int stab_path_store(const char *gpu_name, int n, const stab_path_choice *choice);

/* Empties the cache (host only). */
int stab_path_clear(void);

/* Writes every cached entry to a text file (one line per entry: name, n,
 * resident, resident_adjoint, gen_cut, tile_limit, tuned and gen_parts,
 * tab-separated),
 * or reads such a file into the cache; a
 * file with a malformed line is rejected whole (STAB_E_INVAL) and leaves the
 * cache as it was.  Errors: STAB_E_INVAL (path NULL, malformed file),
 * STAB_E_STATE (the file cannot be opened). */
int stab_path_save(const char *path);
int stab_path_load(const char *path);

/* Measures the candidates for n qubits on CUDA device `device` now, stores
 * the result under that GPU's name and writes it to *out (may be NULL).
 * Candidates: n = 4: two parts with gen_cut in {0.50, 0.53, 0.56, 0.59, 0.62}
 * and three parts with gen_cut in {0.43, 0.45, 0.47, 0.49, 0.51} (time of the
 * generators of a 24,000-gate probe); n = 5, 6: resident against streamed for
 * <O> and, separately, for the gradient (2,000-gate probe); n = 7 .. 9: tiles
 * against one launch per pass, for one vector (<O>) and for n vectors (the
 * generators), giving tile_limit = the largest of those launch sizes where
 * tiles won (0 when neither); n <= 3 and n >= 10 have nothing measured and
 * keep the defaults (marked tuned).  Each candidate takes the best of five
 * timed calls; a candidate replaces the default only when it is more than 2 %
 * faster, so timing noise does not flip a choice.  Takes up to about a tenth
 * of a second.
 * Errors: STAB_E_RANGE (n), STAB_E_CUDA, STAB_E_NOMEM. */
int stab_path_tune(int device, int n, stab_path_choice *out);

/* The choice a context runs with (the defaults for kernels other than AUTO). */
int stab_path_current(stab_ctx *ctx, stab_path_choice *out);

/* ---------------------------------------------------------------- FP64 peak */
/* Measures the FP64 rate of the current device, the roofline of the rotation
 * passes (three FMAs per rotated pair on data that stays on chip, so the FP64
 * pipe, not HBM, bounds them; Sec. II-A's per-gate work).  kind 0: every
 * thread of a full-occupancy grid runs eight independent DFMA chains; kind 1:
 * every warp runs four independent chains of the 8x8x4 FP64 matrix
 * instruction.  iters: chain steps per thread (1 .. 2^30; about 8192 gives a
 * launch of a few tens of milliseconds on a GB300).  One untimed warm-up
 * launch, then one launch timed with CUDA events on a stream the call creates.
 * *tflops receives the achieved TFLOP/s (2 flops per FMA), *ms (may be NULL)
 * the timed launch's duration.  Allocates 2 KiB of device memory for the
 * duration of the call.  Errors: STAB_E_INVAL (kind, tflops NULL),
 * STAB_E_RANGE (iters), STAB_E_CUDA. */
int stab_probe_fp64(int kind, int64_t iters, double *tflops, double *ms);

/* Latency of the pieces of the n = 4 register pass loop (the loop a lone
 * vector of a split generator sweep runs), on one CTA of the current device,
 * by the SM's cycle counter.  A wire pass here is three shuffles that gather
 * a lane's group (I, X, Y, Z slots of one wire in a warp's lanes) and the
 * three dependent FP64 instructions of its row of a 3x3 rotation (Sec. III,
 * the per-wire map of Rx, Ry, Rz); the map is orthogonal, so values stay
 * bounded.  pattern 0: `passes` wire passes, one vector entry per thread;
 * 1: plus a switch of the register layout through shared memory (write, one
 * barrier, read) before every second pass; 2: plus a pull through a
 * four-CNOT ring (Table I), walked record by record, at every fourth pass;
 * 3 (threads = 128): two entries per thread, three register passes and one
 * shared-memory pass merged with the ring's pull per four passes; 4: two-wire
 * fused passes (each 16-entry block of two wires through (1+M) (x) (1+M): up
 * to nine products per output, counted as two wire passes).  threads:
 * 256 (a 4^4 vector) or 128.  passes: a multiple of 4 in [4, 2^24].  Writes
 * the cycles per pass to *clk_per_pass.  Allocates under 3 KiB of device
 * memory for the call.  Errors: STAB_E_INVAL (pattern, threads, NULL),
 * STAB_E_RANGE (passes), STAB_E_CUDA. */
int stab_probe_pass(int pattern, int threads, int64_t passes, double *clk_per_pass);

#ifdef __cplusplus
}
#endif

#endif /* STAB_LIB_INTERFACE_H */
