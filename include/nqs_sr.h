/*
 * nqs_sr.h -- C ABI of the block-layer stochastic-reconfiguration (SR) step
 * for complex neural quantum states, hand-written CUDA for sm_103a (GB300).
 *
 * The step (Sec. 2 of "When Less is More: Approximating the Quantum Geometric
 * Tensor with Block Structures", arXiv 2510.08430):
 *   O_{s,k}  = d ln psi(x_s) / d theta_k                (definition below Eq. 2)
 *   E_loc(x) = <x|H|psi> / <x|psi>                       (Eq. 1)
 *   dO = O - <O>,  e = E_loc - <E>                        (second form of Eq. 2)
 *   F_k = <conj(dO_k) e>                                  (Sec. 2: F = energy gradient)
 *   S_b = <dO_b^H dO_b>  for each layer block b            (Eq. 3)
 *   dtheta_b = -eta * pinv(S_b + lambda I) F_b             (Sec. 2, block-layer paragraph)
 * Expectations <f> = sum_s w_s f(x_s), with w_s = 1/n_s unless weights are given.
 *
 * Conventions used by every call
 * ------------------------------
 * - Complex numbers are interleaved (re, im). "c128" = two doubles, "c64" = two floats.
 * - Unless stated otherwise a pointer argument is a DEVICE pointer owned by the
 *   caller; the library never frees or retains it after the call returns.
 * - The library allocates no device memory. Scratch comes from a caller-provided
 *   workspace (nqs_workspace_create), sized by the *_workspace_size queries.
 * - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *   is the legacy default stream) and returns an int status. Host-side argument
 *   errors and launch failures are returned directly. Device-detected errors
 *   (non-finite values, sweep limits, wait budgets) are recorded in the
 *   workspace and returned by nqs_sync_status, which synchronises `stream`.
 * - No C++ exception, abort or device trap crosses this boundary.
 * - Thread safety: distinct workspaces may be used concurrently from different
 *   host threads; one workspace must not be used by overlapping calls.
 */
#ifndef NQS_SR_H
#define NQS_SR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NQS_API __attribute__((visibility("default")))
#else
#define NQS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define NQS_OK                 0
#define NQS_ERR_INVALID_ARG   (-1) /* bad sizes, offsets, dtype/precision combination, NULL */
#define NQS_ERR_CUDA          (-2) /* a CUDA runtime call or kernel launch failed */
#define NQS_ERR_WORKSPACE     (-3) /* workspace too small; nqs_last_error states the size */
#define NQS_ERR_NOT_CONVERGED (-4) /* an iterative eigen-solver step hit its sweep limit */
#define NQS_ERR_TIMEOUT       (-5) /* a device-side wait exhausted its iteration budget */
#define NQS_ERR_NONFINITE     (-6) /* NaN/Inf found in O, E_loc, S or the solve */
#define NQS_ERR_UNSUPPORTED   (-7) /* valid request this build does not implement */
#define NQS_ERR_RETRY         (-8) /* NQS_GRAPH step whose mixed-solver certificate failed:
                                      retake it without NQS_GRAPH (the FP64 path then runs) */

/* ---- precision of the sample-space contractions (Jacobian, E_loc, Gram) ----
 * NQS_FP64        : everything in FP64 (O is c128), except that the local energies' FFNN
 *                   hidden layers (products and ln cosh of the connected forwards) use
 *                   double-float arithmetic (pairs of FP32 numbers, about 2^-46 relative).
 * NQS_FP32        : Jacobian and E_loc in FP32 (O is c64), centring and force
 *                   accumulated in FP64, Gram in FP32 FFMA.
 * NQS_SPLIT_BF16  : Jacobian and E_loc in FP64 (O is c128), and the Gram on
 *                   tcgen05 tensor cores: every centred entry is split x = hi + lo
 *                   (BF16 roundings of x and of the remainder) and three products
 *                   (hi*hi, hi*lo, lo*hi) are accumulated in FP32 over one
 *                   64-sample block at a time; the blocks are summed in
 *                   double-float. Entry representation error 2^-17. A reduced-accuracy
 *                   mode: its dtheta bar is 1e-2 relative (it misses the 1e-6 bar of the
 *                   split path on the 10x10 lattice; NQS_SPLIT_BF16_EXACT meets it).
 * NQS_SPLIT_BF16X3: as NQS_SPLIT_BF16 with hi + mid + lo and six products
 *                   (all terms above 2^-16 relative): representation error 2^-25.
 * NQS_SPLIT_BF16_EXACT: error-free split on the tensor cores: for every parameter and
 *                   every group of 32 samples the centred values are scaled by a common
 *                   power of two and split into five BF16 slices holding integers of at
 *                   most 8 bits, so that the MMA sums of the leading products are exact;
 *                   fifteen products (every term above 2^-32 of the group scale) per group,
 *                   groups summed in double-float. Better than FP32 rounding of the data
 *                   even on heavy-tailed Jacobian rows.
 * Local energies in the split modes are those of NQS_FP64 unless the flag NQS_ELOC_DIFF32
 * (below) is given. The per-block shifted eigen-decomposition and solve is selected
 * separately (solver argument, below). */
typedef enum {
    NQS_FP64 = 0, NQS_FP32 = 1, NQS_SPLIT_BF16 = 2, NQS_SPLIT_BF16X3 = 3, NQS_SPLIT_BF16_EXACT = 4
} nqs_precision;

/* NQS_ELOC_DIFF32 (flag of sr_step, sr_step_batched and nqs_local_energy_ex; any precision
 * but NQS_FP32): FFNN local energies by FP32 difference propagation. For every connected
 * configuration x' the changes of the pre-activations dz and of the hidden units
 * dh = lncosh(z + dz) - lncosh(z) = log1p(2 sinh(dz/2) (sinh(dz/2) + cosh(dz/2) tanh z))
 * relative to the parent sample x (z and tanh z from its FP64 forward) are carried through
 * the layers in FP32, following the ln cosh branch of the exact forward, so that
 * ln psi(x') - ln psi(x) carries FP32 rounding of the differences only; the rare connections
 * whose branch or range FP32 cannot decide are recomputed in the NQS_FP64 arithmetic. The
 * per-sample error is about 1e-8 of |E_loc| (heavy-tailed, up to ~1e-6). Its effect on
 * dtheta scales with that error over the spread of E_loc across the samples: small when the
 * local energies fluctuate by more than ~1e-3 of their size (the J1-J2 lattices with shallow
 * FFNNs: rms error / spread below 5e-7), too large for states whose E_loc is nearly constant
 * (deep random networks: 1e-4 and more), which need the default arithmetic. RBMs and
 * one-layer networks always take the NQS_FP64 arithmetic. */
#define NQS_ELOC_DIFF32 8

enum { NQS_RBM = 0, NQS_FFNN = 1, NQS_VIT = 2 };

/* Network description (host struct; host pointer `widths`).
 * RBM : widths = {N, M}; ln psi = sum_i a_i x_i + sum_j lncosh(b_j + sum_i W_ji x_i);
 *       parameter layout [a (N) | b (M) | W (M x N row-major)]; 3 blocks.
 * FFNN: widths = {N, h_1, ..., h_{L-1}, 1}; hidden layers z = W h + b, h' = lncosh(z),
 *       last layer linear; layout per layer [W_l (out x in row-major) | b_l]; one
 *       block per layer (Eq. 3: one block per module).
 * VIT : the transformer whose modules define the block partition of Sec. 2 (patching and
 *       embedding, encoder layers, output layer); the paper leaves the network unspecified,
 *       this is a holomorphic variant (complex parameters, no layer norm, position-only
 *       attention). widths = {N, p, d, h} (always four entries), n_layers = number of encoder
 *       layers L >= 0; tokens T = N / p (p divides N), token t = spins t p .. t p + p - 1:
 *         h_t = W_E x_t + b_E;
 *         per encoder layer: u_t = h_t + sum_s A_ts W_V h_s,
 *                            h_t <- u_t + W_2 lncosh(W_1 u_t + b_1) + b_2;
 *         ln psi = w_O . sum_t lncosh(h_t) + b_O.
 *       Layout: [W_E (d x p) | b_E (d)], then per encoder layer [A (T x T) | W_V (d x d) |
 *       W_1 (h x d) | b_1 (h) | W_2 (d x h) | b_2 (d)], then [w_O (d) | b_O (1)]: L + 2 blocks.
 *       FP64 only (NQS_FP64 and the split precisions, whose Jacobian and local energies are
 *       FP64); NQS_FP32 is NQS_ERR_UNSUPPORTED. Limits: T <= 64, d <= 128, h <= 256,
 *       T (3 d + h) <= 6144.
 * lncosh(z) = s z - ln 2 + log1p(exp(-2 s z)), s = sign(Re z) (s = +1 at Re z = 0).
 * Limits of this build: N <= 1024, every width <= 512, n_layers <= 32. */
typedef struct {
    int32_t kind;           /* NQS_RBM, NQS_FFNN or NQS_VIT */
    int32_t n_layers;       /* number of weight layers (RBM: 1) = len(widths) - 1; VIT: encoder layers */
    const int32_t* widths;  /* HOST array of n_layers + 1 entries (VIT: 4) */
} nqs_model;

/* Spin Hamiltonian H = c * sum_b J_b (sx_i sx_j + sy_i sy_j + sz_i sz_j) over a bond
 * list (Sec. 3: Heisenberg chain; J1-J2 square lattice). c = 1 is the Pauli
 * normalisation of the energies in Table 2; c = 0.25 is S = sigma/2.
 * sign_rule = -1 multiplies the off-diagonal (exchange) elements by -1.
 * Bonds must have i != j and 0 <= i, j < n_sites. */
typedef struct {
    int32_t n_sites;
    int32_t n_bonds;
    const int32_t* bond_ij; /* DEVICE int32 [n_bonds][2] */
    const double* bond_J;   /* DEVICE float64 [n_bonds] */
    double c;
    int32_t sign_rule;      /* +1 or -1 */
} nqs_hamiltonian;

/* ---- workspace (caller-owned device memory wrapped in a host handle) ---- */
typedef struct nqs_workspace nqs_workspace;

/* Wraps `bytes` of caller-allocated device memory starting at `device_ptr`
 * (256-byte aligned). Allocates only the small host-side handle. */
NQS_API int nqs_workspace_create(void* device_ptr, size_t bytes, nqs_workspace** ws);
NQS_API int nqs_workspace_destroy(nqs_workspace* ws);

/* Synchronises `stream`, returns the first device-detected status recorded in
 * `ws` since the last call (NQS_OK if none) and clears it. */
NQS_API int nqs_sync_status(nqs_workspace* ws, void* stream);

/* Thread-local text of the last error (never NULL). */
NQS_API const char* nqs_last_error(void);

/* ---- workspace sizes ---- */
NQS_API int nqs_jacobian_workspace_size(const nqs_model* m, int64_t n_s, int32_t precision, size_t* bytes);
NQS_API int nqs_local_energy_workspace_size(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h,
                                    int32_t precision, size_t* bytes);
NQS_API int qgt_block_build_workspace_size(int64_t n_s, int64_t n_p, const int64_t* block_off,
                                   int32_t n_blocks, int32_t precision, size_t* bytes);
NQS_API int qgt_block_solve_workspace_size(const int64_t* block_off, int32_t n_blocks, size_t* bytes);
NQS_API int sr_step_workspace_size(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h,
                           const int64_t* block_off, int32_t n_blocks, int32_t precision,
                           size_t* bytes);

/* ---- packed block storage of S ----
 * Block b (n_b = block_off[b+1] - block_off[b]) occupies n_b*n_b c128 elements
 * starting at element sum_{b'<b} n_{b'}^2, row-major, S_b[k][l] at k*n_b + l.
 * Only the lower triangle k >= l is defined; the rest is unspecified. */
NQS_API int64_t qgt_packed_size(const int64_t* block_off, int32_t n_blocks); /* elements */

/* nqs_jacobian -- ln psi and the log-derivative Jacobian (definition below Eq. 2).
 *   theta      : c128 [n_p] parameters (layout of nqs_model).
 *   configs    : int8 [n_s][N], entries +1 / -1, row-major.
 *   logpsi_out : c128 [n_s].
 *   O_out      : PARAMETER-MAJOR Jacobian, O_out[k*ldo + s] = d ln psi(x_s)/d theta_k;
 *                c64 for NQS_FP32, c128 otherwise. ldo >= n_s. Columns n_s..ldo-1
 *                of every row are written with zeros.
 * The derivative is the complex (holomorphic) derivative; no conjugation. */
NQS_API int nqs_jacobian(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
                 int32_t precision, void* logpsi_out, void* O_out, int64_t ldo,
                 nqs_workspace* ws, void* stream);

/* nqs_vjp -- vector-Jacobian product of ln psi: out[k] = sum_s conj(O[k*ldo + s]) g[s],
 * the gradient a reverse-mode framework propagates to theta for an upstream gradient g of
 * ln psi (ln psi is holomorphic in theta). O as written by nqs_jacobian with the same
 * precision (c64 for NQS_FP32, c128 otherwise); g: c128 [n_s]; out: c128 [n_p]. FP64
 * accumulation. No workspace. */
NQS_API int nqs_vjp(const void* O, int64_t ldo, int64_t n_s, int64_t n_p, int32_t precision, const void* g,
            void* out, void* stream);

/* nqs_local_energy -- E_loc(x_s) (Eq. 1) for the Hamiltonian h:
 *   E_loc(x) = c sum_b J_b [ x_i x_j + [x_i != x_j] 2 sign_rule psi(x^{ij})/psi(x) ],
 * x^{ij} = x with spins i and j flipped; connected configurations are visited in
 * bond order. eloc_out: c128 [n_s]. Arithmetic in FP32 for NQS_FP32; otherwise FP64, with
 * the FFNN hidden layers of the connected forwards in double-float (about 2^-46 relative).
 * nqs_local_energy_ex takes flags: 0 or NQS_ELOC_DIFF32 (not with NQS_FP32); other bits are
 * NQS_ERR_INVALID_ARG. Same workspace size. */
NQS_API int nqs_local_energy(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
                     const nqs_hamiltonian* h, int32_t precision, void* eloc_out,
                     nqs_workspace* ws, void* stream);
NQS_API int nqs_local_energy_ex(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
                        const nqs_hamiltonian* h, int32_t precision, int32_t flags, void* eloc_out,
                        nqs_workspace* ws, void* stream);

/* ---- variational Monte Carlo loop (Sec. 1: samples of |psi|^2 by Markov chain Monte Carlo;
 * Sec. 2: the SR update) ----
 * nqs_metropolis -- n_steps exchange-move Metropolis steps on n_chains independent chains.
 * Each step gives every chain one proposal: with its uniforms (u1, u2, u3) it picks the k1-th
 * up spin i, k1 = floor(u1 n_up), and the k2-th down spin j, k2 = floor(u2 n_down) (sites
 * counted in increasing order), and accepts the exchange x' = x with spins i and j flipped
 * when u3 < |psi(x') / psi(x)|^2 (FP64 forwards; the ratio is that of the FP64 local energies'
 * connected configurations). Total S^z of every chain is conserved; the chains sample |psi|^2
 * in their S^z sector. A chain with no up or no down spin does not move.
 *   theta    : c128 [n_p] (device).
 *   configs  : int8 [n_chains][N] (device), updated in place.
 *   uniforms : float64 [n_steps][n_chains][3] (device) in [0, 1), one triple per step and chain;
 *              may be NULL when n_steps = 0.
 *   n_accepted: int64 [1] (device) or NULL: receives the number of accepted moves.
 * nqs_metropolis_workspace_size gives the workspace it needs.
 * nqs_theta_update -- theta += dtheta (c128 [n_p], device), the update of one SR step. */
NQS_API int nqs_metropolis_workspace_size(const nqs_model* m, int64_t n_chains, size_t* bytes);
NQS_API int nqs_metropolis(const nqs_model* m, const void* theta, int8_t* configs, int64_t n_chains,
                           int32_t n_steps, const double* uniforms, int64_t* n_accepted, nqs_workspace* ws,
                           void* stream);
NQS_API int nqs_theta_update(void* theta, const void* dtheta, int64_t n_p, void* stream);

/* nqs_connections -- the integer work of E_loc: for every sample, the bonds with
 * x_i != x_j in bond order. conn_count: int32 [n_s]; conn_offset: int64 [n_s+1]
 * (exclusive prefix sum); conn_bond: int32 [max_conn] receives the bond indices
 * sample-major. *n_conn_out (host) receives the total; it is an error
 * (NQS_ERR_INVALID_ARG) if max_conn is too small. Synchronises `stream`. */
NQS_API int nqs_connections(const int8_t* configs, int64_t n_s, const nqs_hamiltonian* h,
                    int32_t* conn_count, int64_t* conn_offset, int32_t* conn_bond,
                    int64_t max_conn, int64_t* n_conn_out, nqs_workspace* ws, void* stream);

/* qgt_block_build -- means, centring, force and the block-layer QGT (Eq. 2, Eq. 3).
 *   O        : parameter-major Jacobian as written by nqs_jacobian with the same
 *              precision (c64 for NQS_FP32, c128 otherwise), leading dimension ldo.
 *              OVERWRITTEN with the centred dO for NQS_FP64/NQS_FP32; left
 *              unchanged in the split modes.
 *   w        : float64 [n_s] sample weights summing to 1, or NULL for 1/n_s.
 *   block_off: HOST int64 [n_blocks+1], block_off[0] = 0, strictly increasing,
 *              block_off[n_blocks] = n_p.
 *   eloc     : c128 [n_s].
 *   S_packed : c128, qgt_packed_size elements (lower triangles, see above).
 *   F_out    : c128 [n_p], F_k = sum_s w_s conj(dO_sk) e_s.
 *   Omean_out: c128 [n_p] or NULL.   Emean_out: c128 [1] or NULL. */
NQS_API int qgt_block_build(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const double* w,
                    const int64_t* block_off, int32_t n_blocks, const void* eloc,
                    int32_t precision, void* S_packed, void* F_out, void* Omean_out,
                    void* Emean_out, nqs_workspace* ws, void* stream);

/* qgt_block_build_static -- qgt_block_build without a workspace. The paper has no
 * counterpart: this is an interface variant, not a step of the method.
 * It is meant for callers that have no device memory to lend to the library, e.g. a
 * plug-in interface that hands over only its input and output buffers, or a process
 * whose device memory is entirely held by another allocator. The call allocates
 * nothing: its only scratch, the centred local energies e_s (16 bytes per sample),
 * lives in a fixed array in the library's own static device memory.
 *   Arguments, layouts and results are those of qgt_block_build, with two limits:
 *   precision  : NQS_FP64 or NQS_FP32 only (the split modes need n_p-sized planes);
 *                any other value returns NQS_ERR_INVALID_ARG.
 *   n_s        : at most NQS_STATIC_MAX_SAMPLES; larger n_s returns
 *                NQS_ERR_INVALID_ARG before anything is launched.
 * Set-up: every call whose stream is not capturing looks up the device address of the
 * static array on the current device (cudaGetSymbolAddress) and caches it per device; a
 * call during stream capture uses the cached address. So the first call on each device
 * (with that device current) must be made outside any stream capture, and a device reset
 * is picked up by the next uncaptured call. All pointers must belong to the current device.
 * Nothing in the static array has to start at zero: every element is written by the
 * call before it is read.
 * There is no device-side status: a non-finite O or E_loc shows as NaN/Inf in the
 * outputs instead of in nqs_sync_status.
 * Overlapping calls on one device (concurrent streams or host threads) share the one
 * array and race: order them, e.g. on a single stream. */
#define NQS_STATIC_MAX_SAMPLES 65536
NQS_API int qgt_block_build_static(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const double* w,
                           const int64_t* block_off, int32_t n_blocks, const void* eloc,
                           int32_t precision, void* S_packed, void* F_out, void* Omean_out,
                           void* Emean_out, void* stream);

/* ntk_solve -- the sample-space (NTK) form of the full-QGT update, the comparator of the
 * block-layer step (equal to the full-QGT solve by the push-through identity when no
 * eigenvalue is cut):
 *   dtheta = -eta X^H (X X^H + diag_shift I)^{-1} eps,  X = dO / sqrt(N_s), eps = e / sqrt(N_s),
 * dO = O - <O>, e = E_loc - <E>, uniform weights.
 *   O        : c128 parameter-major Jacobian (nqs_jacobian, NQS_FP64), leading dimension
 *              ldo; OVERWRITTEN with dO.
 *   eloc     : c128 [n_s].   dtheta_out: c128 [n_p].   Emean_out: c128 [1] or NULL.
 *   precision: arithmetic of the N_s x N_s Gram (NQS_FP64, or NQS_FP32 with the mixed
 *              solver); the eigen-solve of X X^H + diag_shift I uses the per-block solver
 *              with the relative cutoff `cutoff`.
 *   Workspace: ntk_solve_workspace_size (holds an N_s x N_s complex128 matrix). */
NQS_API int ntk_solve_workspace_size(int64_t n_s, int64_t n_p, int32_t precision, size_t* bytes);
NQS_API int ntk_solve(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const void* eloc, double diag_shift,
              double cutoff, double eta, int32_t precision, void* dtheta_out, void* Emean_out,
              nqs_workspace* ws, void* stream);

/* ---- sample sharding ----
 * A step over N samples split into shards (one per rank, or several on one GPU) needs
 * two exchanges: the global means before centring, and the sum of the shards' S and F.
 * nqs_shard_sums -- osum_out[k] = sum_{s in shard} O[k*ldo + s] (c128 [n_p]) and
 *   esum_out[0] = sum_{s in shard} E_loc(s) (c128 [1]); FP64 accumulation. Summed over
 *   all shards and divided by N they give <O> and <E>. No workspace.
 * qgt_block_build_shard -- a shard's part of qgt_block_build. Osum_in (c128 [n_p]) and
 *   Esum_in (c128 [1]) are the sums of nqs_shard_sums over ALL shards (the all-reduced
 *   sums), n_total the number of samples over all shards. The library forms the global means
 *   <O> = Osum_in / n_total, <E> = Esum_in / n_total (copied to Omean_out, c128 [n_p], and
 *   Emean_out, c128 [1], when not NULL) and, with weight 1/n_total for every sample,
 *     S_packed = sum_{s in shard} dO_s^H dO_s / n_total (lower triangles, as qgt_block_build),
 *     F_out    = sum_{s in shard} conj(dO_s) e_s / n_total,
 *   dO = O - <O>, e = E_loc - <E>. The sums over all shards of S_packed and F_out are
 *   qgt_block_build's S and F of all N samples. O is overwritten with dO in the
 *   FP64/FP32 modes (as qgt_block_build). n_total < n_s is NQS_ERR_INVALID_ARG.
 *   Workspace: qgt_block_build_workspace_size. */
NQS_API int nqs_shard_sums(const void* O, int64_t ldo, int64_t n_s, int64_t n_p, int32_t precision,
                   const void* eloc, void* osum_out, void* esum_out, void* stream);
NQS_API int qgt_block_build_shard(void* O, int64_t ldo, int64_t n_s, int64_t n_p, int64_t n_total,
                          const int64_t* block_off, int32_t n_blocks, const void* eloc,
                          const void* Osum_in, const void* Esum_in, int32_t precision,
                          void* S_packed, void* F_out, void* Omean_out, void* Emean_out,
                          nqs_workspace* ws, void* stream);

/* ---- per-block solver ----
 * NQS_SOLVE_FP64 : the Householder reduction, eigenvalues and solve all in FP64.
 * NQS_SOLVE_MIXED: the O(n^3) reduction runs in FP32 on a copy of S_b (FP64 units run
 *                  at 1/64 of the FP32 rate on GB300); Q is formed explicitly in FP32;
 *                  eigenvalues come from the FP32-reduced tridiagonal; dtheta_b is then
 *                  obtained by iterative refinement whose residuals F - (S_b + lambda I) x
 *                  use the FP64 S_b, until ||r|| <= 1e-14 ||F_b||. When the FP32
 *                  eigenvalues cannot certify that the cutoff keeps every eigenvalue of a
 *                  block (margin 4e-5 sigma_max), or a block's refinement has not converged
 *                  after 30 sweeps, every block is solved by the FP64 path instead; each
 *                  decision synchronises the stream once (under NQS_GRAPH either is recorded
 *                  as NQS_ERR_RETRY). S_packed is left unchanged in the refinement case.
 * NQS_SOLVE_MIXED_PSD: as NQS_SOLVE_MIXED, with the caller asserting that every S_b is
 *                  a Gram matrix (positive semi-definite up to a rounding of at most
 *                  1e-6 sigma_max, as qgt_block_build produces), so sigma_min >= shift -
 *                  1e-6 sigma_max certifies the cutoff. sr_step uses this certificate when
 *                  called with NQS_SOLVE_MIXED.
 *                  When no eigenvalues are requested (evals_out NULL) and every block has at
 *                  most 65536 parameters, the cutoff is first certified without an
 *                  eigen-decomposition: sigma_max(S~_b) <= ||S_b||_F + shift, sigma_min(S~_b)
 *                  >= shift - 1e-6 ||S_b||_F, and every eigenvalue is kept when the lower bound
 *                  exceeds cutoff * upper bound (relative mode) or cutoff (absolute mode).
 *                  Certified blocks are then solved as the positive-definite system
 *                  S~_b x = F_b: FP32 tiled Cholesky of S~_b and FP64-residual iterative
 *                  refinement until ||F - S~ x|| <= 1e-14 ||F|| (1e-12 ||F|| inside sr_step and
 *                  sr_step_batched in the split precisions, whose S carries ~1e-10 relative
 *                  error of its own), or until the residual stops contracting within 1e-12
 *                  ||F||; dtheta_b = -eta x equals the
 *                  pseudo-inverse update up to rounding. A block that is not certified, meets
 *                  a non-positive FP32 pivot or does not converge sends every block to the
 *                  eigen-decomposition path above (one more host synchronisation); under
 *                  NQS_GRAPH that is recorded as NQS_ERR_RETRY instead. */
enum { NQS_SOLVE_FP64 = 0, NQS_SOLVE_MIXED = 1, NQS_SOLVE_MIXED_PSD = 2 };

/* qgt_block_solve -- per-block shifted pseudo-inverse solve (Sec. 2):
 *   S~_b = S_b + diag_shift I = U diag(sigma) U^H (FP64),
 *   keep_i = sigma_i > cutoff * max_i sigma_i   (cutoff_mode 0, relative)
 *          = sigma_i > cutoff                   (cutoff_mode 1, absolute),
 *   dtheta_b = -eta U diag(keep / sigma) U^H F_b.
 * The eigen-decomposition is kept factored: S~_b = Q (T + diag_shift I) Q^H by
 * Householder reduction (Q stored as reflectors in S_packed, which is
 * OVERWRITTEN), and T = Z diag(sigma) Z^T; Z is formed only when some sigma_i
 * is dropped. The result equals the definition up to rounding.
 *   F         : c128 [n_p].             dtheta_out: c128 [n_p].
 *   evals_out : float64 [n_p] or NULL; block b's sigma ascending at block_off[b].
 *   n_kept_out: int32 [n_blocks] or NULL. */
NQS_API int qgt_block_solve(void* S_packed, const int64_t* block_off, int32_t n_blocks, const void* F,
                    double diag_shift, double cutoff, int32_t cutoff_mode, double eta, int32_t solver,
                    void* dtheta_out, double* evals_out, int32_t* n_kept_out,
                    nqs_workspace* ws, void* stream);

/* sr_step -- one whole block-layer SR step: Jacobian, E_loc, centring, force,
 * block Gram and the per-block solve, from (theta, configs) to dtheta and <E>.
 *   solver: NQS_SOLVE_FP64 or NQS_SOLVE_MIXED (see qgt_block_solve).
 *   dtheta_out: c128 [n_p]; Emean_out: c128 [1].
 *   evals_out / n_kept_out as in qgt_block_solve (may be NULL).
 *   flags: NQS_SYNC makes the call synchronise and return device status.
 *          NQS_PARAM_SPACE solves every block in parameter space (see below).
 *          NQS_ELOC_DIFF32 computes FFNN local energies by FP32 difference propagation
 *          (see above).
 *          NQS_GRAPH makes the call capturable into a CUDA graph (stream capture):
 *          nothing synchronises with the host. The mixed solver's certificate is then
 *          checked on the device; when it fails the step's dtheta is not the definition's
 *          and NQS_ERR_RETRY is recorded in the workspace status (nqs_sync_status). Stage
 *          timing is not recorded, and NQS_SYNC must not be combined with it. The first
 *          call on a device and shape should be made without capture (it sets kernel
 *          attributes and loads kernels). */
#define NQS_SYNC 1
#define NQS_GRAPH 2
#define NQS_PARAM_SPACE 4
/* Blocks wider than the sample count. With the mixed solver, diag_shift > 0, precision
 * NQS_FP64 or NQS_SPLIT_BF16_EXACT and no NQS_PARAM_SPACE flag, a block with n_b > n_s is
 * solved in sample space (push-through identity):
 *   dtheta_b = -eta X_b^H pinv(X_b X_b^H + diag_shift I) eps,  X_b = dO_b / sqrt(n_s), eps = e / sqrt(n_s),
 * with an n_s x n_s Gram (tensor cores in the split precision) in place of the n_b x n_b S_b,
 * and the same cutoff rule; this equals the block's pseudo-inverse update (F_b = X_b^H eps lies
 * in the range of S_b, where S_b + diag_shift I and X_b X_b^H + diag_shift I share their
 * eigenvalues). n_kept_out counts the eigenvalues of S_b + diag_shift I as usual. evals_out
 * must be NULL for such a step (NQS_ERR_UNSUPPORTED otherwise). sr_step_workspace_size2
 * sizes the workspace of any sr_step call (it equals sr_step_workspace_size when no block is
 * solved in sample space). */
NQS_API int sr_step_workspace_size2(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h,
                                    const int64_t* block_off, int32_t n_blocks, double diag_shift, int32_t precision,
                                    int32_t solver, int32_t flags, size_t* bytes);
NQS_API int sr_step(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
            const nqs_hamiltonian* h, const int64_t* block_off, int32_t n_blocks,
            double diag_shift, double cutoff, int32_t cutoff_mode, double eta,
            int32_t precision, int32_t solver, void* dtheta_out, void* Emean_out, double* evals_out,
            int32_t* n_kept_out, int32_t flags, nqs_workspace* ws, void* stream);

/* sr_step_batched -- n_inst independent SR steps in one call (batching of many
 * instances). Instance i has its own model, n_s[i] samples, Hamiltonian and block
 * partition; diag shift, cutoff, eta, precision and solver are shared. The Jacobians,
 * local energies and centring run per instance; in the split precisions all blocks of
 * all instances share one grouped tensor-core Gram launch (sample axis zero-padded to
 * the largest n_s, which adds nothing), and every block goes through one eigensolver
 * launch. Results equal n_inst separate sr_step calls up to rounding.
 *   models[n_inst], hams[n_inst], n_s[n_inst], n_blocks[n_inst]: HOST arrays.
 *   theta     : c128, the instances' parameter vectors concatenated.
 *   configs   : int8, the instances' configuration arrays concatenated.
 *   block_off : HOST int64, per instance its n_blocks[i] + 1 offsets (each starting at
 *               0 and ending at that instance's n_p), concatenated.
 *   dtheta_out: c128 [sum n_p], concatenated; Emean_out: c128 [n_inst].
 *   evals_out : float64 [sum n_p] or NULL; n_kept_out: int32 [sum n_blocks] or NULL.
 * At most 256 blocks over all instances (NQS_ERR_INVALID_ARG beyond). */
NQS_API int sr_step_batched_workspace_size(int32_t n_inst, const nqs_model* models, const int64_t* n_s,
                                   const nqs_hamiltonian* hams, const int64_t* block_off,
                                   const int32_t* n_blocks, int32_t precision, size_t* bytes);
NQS_API int sr_step_batched(int32_t n_inst, const nqs_model* models, const void* theta, const int8_t* configs,
                    const int64_t* n_s, const nqs_hamiltonian* hams, const int64_t* block_off,
                    const int32_t* n_blocks, double diag_shift, double cutoff, int32_t cutoff_mode,
                    double eta, int32_t precision, int32_t solver, void* dtheta_out, void* Emean_out,
                    double* evals_out, int32_t* n_kept_out, int32_t flags, nqs_workspace* ws,
                    void* stream);

/* ---- inverse-metric diagnostics (Eq. 4; Sec. 3, Table 1) ----
 * nqs_born_weights -- w_out[s] = |psi(x_s)|^2 / sum_t |psi(x_t)|^2 from logpsi (c128 [n]):
 *   the sample weights that turn an enumeration of all 2^N configurations into exact
 *   expectations (qgt_block_build with these weights gives the exact QGT). float64 [n] out.
 * qgt_inverse_diagnostics -- with A = pinv(S_a' + diag_shift I) and B = pinv(S_b + diag_shift I),
 *   S_a' the restriction of S_a to the diagonal blocks of block_off_a (the block-layer QGT of
 *   a full QGT; n_blocks_a = 1 keeps all of S_a), and the cutoff rule of qgt_block_solve:
 *     out[0] = F(A, B)     = Tr[A^H B] / (|A|_F |B|_F)            (Frobenius overlap)
 *     out[1] = eps_F(A, B) = |A - B|_F / |B|_F                     (relative Frobenius error)
 *     out[2] = kappa(A), out[3] = kappa(B): largest over smallest kept eigenvalue
 *     out[4] = r_lambda(A, B): Pearson correlation of the spectra of A and B, each in
 *              descending order (eigenvalues cut by the pseudo-inverse count as 0).
 *   S_a, S_b: c128 n x n row-major, lower triangle used (DEVICE); out: DEVICE float64 [5].
 *   FP64 eigen-decompositions with eigenvectors (Householder, implicit QL); n <= 12000.
 *   Workspace: qgt_inverse_diagnostics_workspace_size (about 64 n^2 bytes). */
NQS_API int nqs_born_weights(const void* logpsi, int64_t n, double* w_out, void* stream);
NQS_API int qgt_inverse_diagnostics_workspace_size(int64_t n, size_t* bytes);
NQS_API int qgt_inverse_diagnostics(const void* S_a, const int64_t* block_off_a, int32_t n_blocks_a,
                                    const void* S_b, int64_t n, double diag_shift, double cutoff,
                                    int32_t cutoff_mode, double* out, nqs_workspace* ws, void* stream);

/* ---- measurement hooks ----
 * nqs_stage_timing(ws, 1) makes later sr_step calls on `ws` record CUDA events
 * on their stream at the stage boundaries: [0] Jacobian (parameter conversion,
 * forward, backward, O write), [1] local energies, [2] means/centring/force,
 * [3] block Gram (plus the solver's set-up copies and, on the Cholesky path, the FP32 tile
 * copy and certificate), [4] factorization: the FP32 tiled Cholesky panels of the Gram-matrix
 * path, or the Householder tridiagonal reduction (exactly its one kernel) of the eigen path,
 * [5] refinement, eigenvalues, solve and back-transform. nqs_stage_times synchronises on the last event and
 * returns the milliseconds of each stage of the most recent timed sr_step.
 * nqs_launch_count returns the number of kernels this library has launched in
 * the process (all threads). */
/* nqs_set_limits -- test hook of the failure paths (process-wide, all devices; takes effect
 * for calls made after it returns). max_sweeps > 0 replaces both the implicit-QL sweep limit
 * per eigenvalue (default 60) and the iterative-refinement sweep limit (default 30); a limit
 * that runs out records NQS_ERR_NOT_CONVERGED. wait_ns > 0 replaces the budget of every
 * device-side wait of the persistent solver kernels (grid barriers, wavefront flags; default
 * 2 s); a wait that runs out records NQS_ERR_TIMEOUT and its kernel returns. 0 restores a
 * default. Results computed under lowered limits are not the definition's. */
NQS_API int nqs_set_limits(int32_t max_sweeps, int64_t wait_ns);

/* nqs_set_eloc_fallback_all -- test hook (process-wide): on != 0 sends every connection of
 * the FP32 difference-propagation local energies (NQS_ELOC_DIFF32) to the FP64-class
 * kernel that otherwise recomputes only the connections FP32 cannot follow, so that this
 * path can be checked on its own; the results are then those of NQS_FP64. 0 restores. */
NQS_API int nqs_set_eloc_fallback_all(int32_t on);

/* ---- tuning of the tensor-core Gram ----
 * The persistent tcgen05 Gram takes the 128 x 128 tiles of each block in square groups of
 * G x G tiles, so that the CTAs running at the same time share G row and G column panels
 * in L2. nqs_set_gram_tuning installs a table (process-wide, at most 64 entries; n = 0
 * clears it): a call whose largest block has at most max_nb[e] parameters and which sums
 * at most max_ns[e] samples uses group[e] (1 <= group <= 64), the first matching entry
 * wins; without a match G = 8. The table is written by the project's tuner
 * (paper_2510_08430_gb300.tune), which times the candidates on the device. The choice changes
 * only the order of the tiles, never the arithmetic: S is bitwise the same for every G.
 * nqs_gram_group_edge returns the G a call with that shape would use. */
NQS_API int nqs_set_gram_tuning(int32_t n, const int64_t* max_nb, const int64_t* max_ns, const int32_t* group);
NQS_API int32_t nqs_gram_group_edge(int64_t max_nb, int64_t n_s);

NQS_API int nqs_stage_timing(nqs_workspace* ws, int32_t enable);
NQS_API int nqs_stage_times(nqs_workspace* ws, double* ms_out, int32_t max_stages, int32_t* n_stages);
NQS_API int64_t nqs_launch_count(void);

/* Library version string. */
NQS_API const char* nqs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NQS_SR_H */
