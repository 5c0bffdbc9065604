/*
 * psatd.h -- C ABI of libpsatd.so, a GB300 (sm_103a) local-FFT PSATD Maxwell
 * solver after Vincenti & Vay, arXiv:1707.08500.
 *
 * The method (Sec. 3.2, Fig. 2a, Fig. 3): the periodic global grid is cut into
 * subdomains; each is padded with n_g guard cells per side; every step each
 * padded box is transformed with a local 3D real FFT, every Fourier mode is
 * advanced analytically in time with Eq. 1a/1b (Sec. 3.1) using the order-p
 * modified wavenumber, the box is transformed back, and the guard cells are
 * replaced by the valid values of the subdomains that own them.
 *
 * Units: c = 1 and eps0 = 1 (Sec. 2, Eq. 2b reads D_t E = curl B - J).
 *
 * Memory model: the caller owns the device memory of the solver (field arenas
 * and one workspace); the library never allocates device memory.  The one
 * exception is the fixed buffer behind psatd_push_static: a file-scope device
 * array of PSATD_STATIC_WORKSPACE_BYTES (32 MiB) that every GPU which loads the
 * library holds from module load until the process exits.  A plan owns only
 * host metadata.  psatd_push, psatd_push_profiled, psatd_exchange_guards and
 * psatd_yee_step only enqueue work on their stream: no synchronisation, no
 * allocation, no host read of device data -- so they may be captured into a
 * CUDA graph.  Pushes of one plan must not overlap on the GPU (they share the
 * plan's workspace; psatd_check reports it).  A plan is not thread-safe;
 * different plans are independent.  psatd_set_workspace and psatd_set_coeffs
 * are set-up calls: they copy metadata and tables to the workspace with
 * blocking copies on the legacy default stream (on the plan's bound stream,
 * synchronised, for plans made with psatd_plan).
 *
 * Errors: every function returns PSATD_OK (0) or a negative status; no C++
 * exception crosses the ABI.  psatd_last_error() gives a human-readable
 * message for the last failing call on a plan.  Kernel launch failures are
 * reported as PSATD_E_CUDA (checked with cudaPeekAtLastError, no sync).
 */
#ifndef PSATD_H
#define PSATD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define PSATD_OK              0
#define PSATD_E_ARG          -1  /* null pointer, bad enum, bad count          */
#define PSATD_E_SHAPE        -2  /* decomposition does not tile the grid, odd p,
                                    guard wider than supported, bad extent    */
#define PSATD_E_NOMEM        -3  /* workspace smaller than psatd_workspace_bytes */
#define PSATD_E_CUDA         -4  /* a CUDA runtime call or launch failed       */
#define PSATD_E_UNSUPPORTED  -5  /* local length not a product of two or three
                                    factors in 1..16, or odd local x length   */
#define PSATD_E_STATE        -6  /* workspace or coefficients not set yet      */
#define PSATD_E_TIMEOUT      -7  /* reserved: a bounded device wait gave up    */

/* ---- plan flags ---------------------------------------------------------- */
#define PSATD_F32            0x01 /* fields, spectra and FFTs in FP32; Eq. 1
                                     coefficient tables built in FP64, stored FP32 */
#define PSATD_F64            0x02 /* everything in FP64                          */
#define PSATD_STAGGERED      0x04 /* Yee-staggered components (not in the paper):
                                     order-p staggered modified wavenumber and
                                     exact-k phase shifts to nodal position     */
#define PSATD_GAUSS_DIAG     0x08 /* read rho and return per-subdomain FP64 sums
                                     of |i[k].E~ - rho~|^2 and |rho~|^2 (partial
                                     sums per work item in the plan's precision,
                                     accumulated in FP64)                        */
#define PSATD_PLAIN          0x10 /* baseline schedule: one subdomain per launch,
                                     guards refilled by a separate exchange
                                     kernel (default: all subdomains batched in
                                     one launch per stage, guard images written
                                     by the inverse-FFT stage itself)            */
#define PSATD_2D             0x40 /* a two-dimensional (x, y) problem: global_n[2]
                                     == 1, every subdomain has n[2] == 1, and
                                     there are no guard cells along z (the
                                     local boxes are Lx x Ly x 1)                */
#define PSATD_GRID_PER_ITEM  0x20 /* launch one CTA per work item instead of the
                                     default persistent grid (as many CTAs as
                                     fit on the GPU, drawing work items from a
                                     counter in the workspace)                   */
#define PSATD_HEAT           0x100 /* the local-FFT heat equation instead of
                                     Maxwell (Sec. 5: the decomposition applies
                                     to other initial-value problems; the
                                     paper names the heat equation).  One scalar
                                     field T in fields->E[0] is advanced per
                                     step by the exact per-mode solution of
                                     dT/dt = D lap T + Q:
                                       T~' = exp(-x) T~ + (1-exp(-x))/x S~,
                                       x = D dt sum_u [k_u]^2,
                                     with [k_u] the order-p staggered modified
                                     wavenumber (p = 0: exact k; the Nyquist
                                     index keeps k = pi/du) and S = Q dt the
                                     heat added per cell over the step.  Not
                                     with PSATD_STAGGERED or PSATD_GAUSS_DIAG. */
#define PSATD_HEAT_SOURCE    0x200 /* with PSATD_HEAT: a source S in
                                     fields->J[0] (read only)                   */
#define PSATD_GENERIC_PLANES 0x400 /* FP32: run every stage with the generic
                                     batched kernels even where the ones with
                                     thread-private transforms of compile-time
                                     length apply (see psatd_plane_engine)     */
#define PSATD_PACKED_Z       0x800 /* FP32: the z/Eq. 1 stage with one thread per
                                     mode pair and quarter of its z DFTs, the
                                     two modes of a pair on packed FP32x2
                                     lanes, for the local z lengths compiled in
                                     (see psatd_plane_engine).  It executes
                                     fewer instructions than the default
                                     batched z/Eq. 1 kernel but holds fewer
                                     warps per SM, which on 96^3 boxes makes
                                     it slower; opt-in                        */
#define PSATD_SPLIT_PLANES   0x80 /* split-plane schedule: the x and y transforms
                                     of the forward and inverse plane stages run
                                     as separate row and column launches (five
                                     stages per push instead of three).  Chosen
                                     automatically when an (x, y) plane of a
                                     local box does not fit in shared memory
                                     (e.g. one box over the whole grid, the
                                     paper's PSATD-global, Sec. 3.2 / Fig. 2b);
                                     this flag forces it for any plan         */

/* One subdomain.  Its valid cells are the global indices [lo, lo+n) per axis
 * (x, y, z); its local (padded) box is [lo-ng, lo+n+ng), of extent
 * L = n + 2 ng per axis, read modulo the periodic global grid.
 * order: even p >= 2, or 0 for the infinite-order limit (exact k). */
typedef struct {
    int32_t lo[3];
    int32_t n[3];
    int32_t ng;
    int32_t order;
} psatd_sub;

/* Device pointers to the field arenas (one arena per component).  Every
 * subdomain's local box is stored at the offset given by psatd_layout, as a
 * dense [Lz][Ly][Lx] array (x fastest) of float (PSATD_F32) or double
 * (PSATD_F64).  E and B hold the fields at time n on entry and n+1 on return;
 * J (at n+1/2) and rho (at n+1, read only with PSATD_GAUSS_DIAG, else may be
 * NULL) are read only.  Every pointer must be 16-byte aligned. */
typedef struct {
    void*       E[3];
    void*       B[3];
    const void* J[3];
    const void* rho;
} psatd_fields;

typedef struct psatd_plan_s* psatd_plan_t;

/* Build a plan (host only, no CUDA call) for the decomposition of Sec. 3.2
 * (Fig. 2a): the periodic global grid cut into subdomains, each padded with
 * ng guard cells per side, each advanced with its own local FFTs at stencil
 * order p.  global_n: periodic global grid
 * (x, y, z).  Validated: the valid boxes tile the global grid exactly; every
 * order is 0 or even; the local x length is even, and every local length
 * (half of it along x) factors as n1*n2 with 1 <= n1, n2 <= 16, or else as
 * n1*n2*n3 with 2 <= n1, n2, n3 <= 16 (so any length whose prime factors are
 * 2, 3, 5, 7, 11 and 13 with at most three factors per 16, up to 4096; local
 * x up to 8192); flags hold exactly one of PSATD_F32 /
 * PSATD_F64.  Guard widths may exceed a neighbour's width (the guard is then
 * filled from several owners). */
int psatd_plan_create(psatd_plan_t* plan, const int32_t global_n[3],
                      const psatd_sub* subs, int32_t nsub, int32_t flags);

/* psatd_plan_create that also binds a CUDA stream to the plan (a
 * cudaStream_t; NULL = the legacy default stream): the set-up calls
 * psatd_set_workspace and psatd_set_coeffs then enqueue their host-to-device
 * copies on that stream and synchronise it before returning, instead of
 * copying on the legacy default stream.  Pushes still take their own stream
 * argument.  Same validation and status codes as psatd_plan_create. */
int psatd_plan(psatd_plan_t* plan, const int32_t global_n[3], const psatd_sub* subs, int32_t nsub,
               int32_t flags, void* cuda_stream);

/* Tunable launch shapes of a plan (0 = library default for every field).
 * chunk_b: (ky,kx) modes per CTA of the z/Eq. 1 stage, 1..1024 (reduced
 * until the stage's tile fits in shared memory);
 * f1[3]: first factor of the two-stage FFT of the x (half length), y and z
 * axes; used for every subdomain whose length it divides with both factors
 * in 1..16, ignored otherwise (and for axes split in three factors). */
typedef struct {
    int32_t chunk_b;
    int32_t f1[3];
} psatd_tuning;

/* psatd_plan_create with explicit tuning (NULL = defaults). */
int psatd_plan_create_tuned(psatd_plan_t* plan, const int32_t global_n[3], const psatd_sub* subs,
                            int32_t nsub, int32_t flags, const psatd_tuning* tuning);

/* Offset (in elements) of subdomain `sub` in every field arena, and its local
 * extents (x, y, z): the padded local box of Sec. 3.2 / Fig. 2a, valid extent
 * plus ng guard cells on each side.  Any output pointer may be NULL. */
int psatd_layout(psatd_plan_t plan, int32_t sub, int64_t* offset_elems, int32_t local_n[3]);

/* Number of elements each field arena must hold. */
int psatd_arena_elems(psatd_plan_t plan, int64_t* elems);

/* Bytes of device workspace the plan needs (spectra, coefficient tables,
 * twiddles, descriptors, partial sums). */
int psatd_workspace_bytes(psatd_plan_t plan, size_t* bytes);

/* Attach caller-owned device workspace (256-byte aligned, at least
 * psatd_workspace_bytes) and copy the plan's device metadata into it.  The
 * memory stays owned by the caller and must outlive the plan's use. */
int psatd_set_workspace(psatd_plan_t plan, void* dev_ptr, size_t bytes);

/* Build the Eq. 1 coefficient tables (C, S, S/k, 1-C, (1-C)/k, S/k - dt, 1/k
 * per mode, order-p modified wavenumbers, stagger phases, FFT twiddles) in
 * FP64 on the host for c_dt = c*dt and cell sizes dx (x, y, z), and copy them
 * to the workspace (rounded to FP32 for PSATD_F32).  Tables are shared by all
 * subdomains with the same local shape and order.  Requires the workspace. */
int psatd_set_coeffs(psatd_plan_t plan, double c_dt, const double dx[3]);
/* For PSATD_HEAT plans the scalar argument is D*dt instead of c*dt, and the
 * tables hold exp(-x) and (1-exp(-x))/x per mode. */

/* One PSATD step of every subdomain (Sec. 3.2 with Eq. 1), followed by the
 * guard replacement (Fig. 3 step 3), enqueued on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  E, B are updated in place.  On entry the
 * guard cells must hold the owners' values (call psatd_exchange_guards once
 * after loading the initial valid fields); on return they do again.
 * gauss_dev: NULL, or a device array of 2*nsub doubles that receives, per
 * subdomain, sum |i[k].E~^{n+1} - rho~|^2 and sum |rho~|^2 over the full
 * spectrum of its padded box (unnormalised transforms); requires
 * PSATD_GAUSS_DIAG. */
int psatd_push(psatd_plan_t plan, const psatd_fields* fields, double* gauss_dev, void* stream);
/* PSATD_HEAT plans: the same step for the scalar T (fields->E[0], updated in
 * place, guards included) with the optional source fields->J[0]; every other
 * pointer of `fields` is ignored and gauss_dev must be NULL. */

/* psatd_push that also records caller-created CUDA events on `stream` at the
 * stage boundaries of the batched schedule: events[0] before pass A (forward
 * x/y), events[1] after pass A, events[2] after pass B (z transforms and
 * Eq. 1), events[3] after pass C (inverse y/x and guard images).  Any entry
 * may be NULL.  With PSATD_PLAIN only events[0] and events[3] are recorded.
 * Used to time each stage inside a running loop. */
int psatd_push_profiled(psatd_plan_t plan, const psatd_fields* fields, double* gauss_dev, void* stream,
                        void* const events[4]);

/* Size of the device buffer behind psatd_push_static (32 MiB). */
#define PSATD_STATIC_WORKSPACE_BYTES (32u * 1024u * 1024u)

/* psatd_push for callers that cannot allocate device memory.  (The paper has
 * no counterpart; this is a convenience of the library.)  Some callers may
 * not call cudaMalloc: a plugin hosted by an application that owns every
 * device allocation and gives it no allocator, or a code path where a
 * cudaMalloc -- which can synchronise the whole device -- is not allowed.
 * Such callers still pass their field arenas and optional Gauss output, but
 * no workspace: the push runs the same kernels on a workspace held in one
 * library-owned, file-scope device array of PSATD_STATIC_WORKSPACE_BYTES that
 * every GPU which loads the library keeps until the process exits.
 *
 * c_dt and dx are the parameters otherwise given to psatd_set_coeffs; the
 * plan needs neither psatd_set_workspace nor psatd_set_coeffs.  Plans whose
 * psatd_workspace_bytes exceeds PSATD_STATIC_WORKSPACE_BYTES are rejected
 * with PSATD_E_NOMEM.  Each call first copies the plan's descriptors and
 * Eq. 1 tables into that array (stream-ordered on `stream`), then enqueues
 * the stages; it allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  Every call and every plan share the one array per
 * device, which keeps the last call's contents: each call rewrites
 * everything its kernels read before they read it (the ticket counters are
 * set to zero); only the device error word is kept across calls, for
 * psatd_check on a plan without a workspace (it starts at zero when the
 * library is loaded and psatd_check clears it).  Calls that overlap on the GPU (different streams or threads
 * without ordering) race on the array.  The first call on each device looks
 * the array's device address up once (with that device current); make that
 * first call before any stream capture.  A call on a device whose context was
 * reset after that lookup is not supported. */
int psatd_push_static(psatd_plan_t plan, double c_dt, const double dx[3], const psatd_fields* fields,
                      double* gauss_dev, void* stream);

/* Global arrays <-> padded-box arenas (the layout of Sec. 3.2 / Fig. 2a).
 * psatd_scatter_global fills every local cell of every subdomain's box --
 * valid cells and guard images, read by global index modulo the periodic
 * grid -- of arenas[f] from global_in[f], for f < nfields (1..10); the result
 * is what psatd_push expects on entry, so no exchange is needed after it.
 * psatd_gather_global writes each box's valid cells of arenas[f] into
 * global_out[f].  Global arrays are dense device arrays [Nz][Ny][Nx] and
 * arenas are psatd_arena_elems long, both of the plan's precision, owned by
 * the caller, aligned to the element size; sources and destinations must not
 * overlap.  Enqueued on `stream`, no allocation; needs the workspace (its copy
 * descriptors are uploaded by psatd_set_workspace). */
int psatd_scatter_global(psatd_plan_t plan, const void* const* global_in, void* const* arenas, int32_t nfields,
                         void* stream);
int psatd_gather_global(psatd_plan_t plan, const void* const* arenas, void* const* global_out, int32_t nfields,
                        void* stream);

/* Introspection of the coefficient tables (host only, no CUDA call): the
 * real table image psatd_set_coeffs would upload for (c_dt, dx), in the
 * plan's precision.  For one table set (the subdomains sharing a local shape,
 * order and FFT factorisation, in order of first use), 7 arrays of
 * Lz*Ly*(Lx/2+1) values -- C, S, S/k, 1-C, (1-C)/k, S/k - dt (all scaled by
 * 1/(Lx Ly Lz)) and 1/k -- in the position order of the forward transforms,
 * padded to 64 elements, then [k] of the x (Lx/2+1), y and z positions, padded
 * to 64.  out == NULL: *bytes receives the size. */
int psatd_debug_tables(psatd_plan_t plan, double c_dt, const double dx[3], void* out, size_t* bytes);

/* Introspection of the guard exchange (Fig. 3 step 3) the plan built (host
 * only).  *count receives the number of copy segments; if segs is not NULL it
 * receives 12 int32 per segment: source subdomain, destination subdomain,
 * first source local cell (x, y, z), extents (x, y, z), offset from source
 * local to destination local coordinates (x, y, z), and 1 for a subdomain's
 * own valid box (0 for a guard image).  Every local cell of every box is the
 * destination of exactly one segment cell. */
int psatd_exchange_segments(psatd_plan_t plan, int32_t* count, int32_t* segs);

/* The guard replacement of Fig. 3 step 3 (Sec. 3.2) on its own: copy every
 * valid cell into each guard cell that images it (all 26
 * neighbour directions, periodic wrap), for E and B only (T only for
 * PSATD_HEAT plans), on `stream`. */
int psatd_exchange_guards(psatd_plan_t plan, const psatd_fields* fields, void* stream);

/* Release the plan's host memory (the workspace stays the caller's). */
int psatd_destroy(psatd_plan_t plan);

/* Static text of a status code. */
const char* psatd_status_string(int status);

/* Message of the last failing call on `plan` ("" if none; valid until the
 * next call on the plan). */
const char* psatd_last_error(psatd_plan_t plan);

/* Which stage kernels the plan uses: the index of the compiled fixed
 * geometry (every subdomain the same cubic box with default FFT splits:
 * FP32 sides 96/64/48/32 with 16/16/8/0 guards, FP64 96/48/32 with 16/8/0),
 * -2 for the kernels that read the geometry from each descriptor with the
 * default z/Eq. 1 chunk width (8 modes FP32, 4 FP64) compiled in, or -1 for
 * the fully descriptor-driven kernels. */
int psatd_geometry_variant(psatd_plan_t plan, int32_t* variant);

/* Which kernels run the stages, as bits: 1 -- the forward (x, y) and inverse
 * (y, x) plane stages are FP32 kernels in which one thread transforms a whole
 * row and a thread a column pair, with the DFT bodies unrolled for the local
 * lengths compiled in (x: 32, 40, 48, 56, 64, 72, 88, 96, 104; y: 32, 48, 64,
 * 80, 96; default factorisations; not with the split-plane schedule);
 * 2 -- the z/Eq. 1 stage is the packed FP32 kernel (PSATD_PACKED_Z) for
 * the local z lengths compiled in (32, 48, 64, 80, 96; default
 * factorisation; an even number of modes per plane; 6 modes per work item;
 * not for PSATD_HEAT).
 * 0 -- the generic batched kernels throughout.  PSATD_GENERIC_PLANES turns
 * both off. */
int psatd_plane_engine(psatd_plan_t plan, int32_t* engine);

/* Number of kernel launches one psatd_push enqueues for this plan. */
int psatd_push_launches(psatd_plan_t plan, int32_t* launches);

/* Debug helper: synchronises the device, then returns and clears the plan's
 * device error word (in its attached workspace; for a plan without one, in
 * the static workspace of its last psatd_push_static -- a word shared by all
 * static pushes on that device; PSATD_E_STATE if the plan has neither).
 * Bits: PSATD_CHECK_ITEM -- a work item was decoded outside its subdomain's
 * item range (the workspace's descriptors were overwritten);
 * PSATD_CHECK_TICKETS -- a persistent launch drew more tickets than it
 * issues, i.e. two pushes of the plan overlapped on the GPU (their results
 * are then undefined).  Kernels set bits and carry on; they never wait. */
#define PSATD_CHECK_ITEM     0x1
#define PSATD_CHECK_TICKETS  0x2
#define PSATD_CHECK_WAIT     0x4  /* a bounded wait for a bulk copy into shared
                                     memory gave up; the CTA stopped early    */
int psatd_check(psatd_plan_t plan, int32_t* error_bits);

#ifdef __cplusplus
}
#endif
#endif /* PSATD_H */
