/*
 * cvq.h -- C-ABI of the GB300 (sm_103a) CV-ADAPT-VQE hot-path library, libcvq.so.
 *
 * The library simulates qumode ansatz circuits on a Fock space truncated to
 * D levels per mode and restricted to the Hamiltonian's symmetry sector
 * (arXiv 2606.05297):
 *   - Bose-Hubbard (Eq. BoseHubbard, Sec. III.A): fixed total boson number N,
 *     D = N + 1 (exact truncation, Sec. III.A);
 *   - bosonic Kitaev chain with optional Kerr term (Eqs. BosonicKitaevChain,
 *     BosonicKitaevChain_Kerr, Sec. III.B): fixed global parity, cutoff d.
 *
 * State vectors are arrays of cvq_c128 (interleaved re, im; the layout of a
 * contiguous complex128 tensor) indexed by the lexicographic rank of the
 * occupation tuple (n_0, ..., n_{L-1}) within the sector, mode 0 most
 * significant.  For Bose-Hubbard that rank is the combinatorial number system
 * of compositions of N; for the Kitaev chain (even d) it is
 * floor(sum_r n_r d^(L-1-r) / 2).
 *
 * Conventions shared by every call:
 *   - Return value: CVQ_OK (0) or an error code; the message of the last error
 *     on the calling thread is cvq_last_error().  Nothing throws across the ABI.
 *   - Pointers named *_dev, psi*, sigma, workspace are DEVICE pointers owned by
 *     the caller (allocated on the current device, 256-byte aligned, not
 *     aliased unless stated).  Pointers without that mark are HOST pointers.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls only enqueue work; results are valid after the stream is
 *     synchronised.  Only cvq_init_sector and cvq_set_pool synchronise.
 *   - Device-side failures are not possible by construction (every index is
 *     derived from a checked sector, and no kernel waits on another); a CUDA
 *     launch or runtime error is reported as CVQ_ECUDA, except an error that
 *     leaves the CUDA context unusable, reported as CVQ_EDEVICE
 *     (cvq_status_from_cuda gives the mapping).
 *   - cvq_sector and cvq_pool are opaque, library-owned, immutable after
 *     creation, and may be shared by concurrent calls on different streams.
 *
 * Limits: 1 <= L <= 16 modes (L >= 2 when periodic); at most 512 pool
 * elements and 512 gates per call; local cutoff D = N + 1 (BH) or d (BKC) with
 * 2 <= D <= 16; BKC requires even d; sector dimension <= 2^40.
 */
#ifndef CVQ_H
#define CVQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } cvq_c128;

enum cvq_status {
    CVQ_OK = 0,
    CVQ_EINVAL = 1,    /* bad argument (sizes, limits, op outside the sector's symmetry) */
    CVQ_ENOMEM = 2,    /* host or device allocation failed */
    CVQ_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed; the context is still usable */
    /* 4 is not used: no call of this library waits on the device with a time limit */
    CVQ_EDEVICE = 5    /* the CUDA context is unusable: some kernel of this process hit a device-side
                          fault (an illegal address or instruction, a failed assertion, an
                          uncorrectable ECC error); every later call fails the same way until the
                          process resets the device */
};

/* The status this library returns for the CUDA runtime error code `cuda_error`
 * (a cudaError_t value): CVQ_OK for cudaSuccess, CVQ_EDEVICE for the errors
 * that leave the context unusable, CVQ_ENOMEM for cudaErrorMemoryAllocation,
 * CVQ_ECUDA otherwise.  Host only; needs no device. */
int cvq_status_from_cuda(int cuda_error);

enum cvq_kind { CVQ_BH = 0, CVQ_BKC = 1 };

/* Pool generator types.  The gate is exp(theta A) (Sec. IV.B, O_r = exp(theta_r A_r))
 * with the anti-Hermitian A below and e^{i phi} = i^phase (phase in 0..3):
 *   HOP      BS(theta, phi), Sec. II.B:  e^{i phi} a_i a_j^dag - e^{-i phi} a_i^dag a_j
 *   SQ2      S2(theta, phi), Sec. II.B:  e^{i phi} a_i a_j - e^{-i phi} a_i^dag a_j^dag
 *   SQ1      S(theta, phi),  Sec. II.B:  (e^{-i phi} a_i^2 - e^{i phi} a_i^dag^2) / 2
 *   PAIRHOP  e^{i phi} a_i^2 a_j^dag^2 - e^{-i phi} a_i^dag^2 a_j^2   (phase 1: i((a_i^dag)^2 a_j^2 + h.c.))
 *   KERR     K(theta) = exp(i theta N^2), Sec. II.B:  A = i n_i^2
 *   NN1      A = i n_i (n_i - 1)
 *   ROT      R(theta) = exp(i theta N), Sec. II.B:  A = i n_i
 *   XKERR    CK(theta) = exp(i theta N_1 N_2), Sec. II.B:  A = i n_i n_j
 * j is ignored for single-mode types.  SQ2 and SQ1 break N and are rejected
 * in a Bose-Hubbard sector (CVQ_EINVAL). */
enum cvq_op_type {
    CVQ_OP_HOP = 0, CVQ_OP_SQ2 = 1, CVQ_OP_SQ1 = 2, CVQ_OP_PAIRHOP = 3,
    CVQ_OP_KERR = 4, CVQ_OP_NN1 = 5, CVQ_OP_ROT = 6, CVQ_OP_XKERR = 7
};

typedef struct { int type, i, j, phase; } cvq_op;

/* Lattice model.  Bonds b = 0..nb-1 join r = b and s = (b + 1) mod L, with
 * nb = L (periodic) or L - 1 (open).  H =
 *     sum_b hop[b] (a_r^dag a_s + a_s^dag a_r) + pair[b] (a_r a_s + a_r^dag a_s^dag)
 *   + sum_r onsite_nn1[r] n_r (n_r - 1) + onsite_n2[r] n_r^2 + onsite_n[r] n_r.
 * Eq. (BoseHubbard): hop = -J, onsite_nn1 = -U/2, onsite_n = -mu.
 * Eq. (BosonicKitaevChain): hop = -J, pair = -Delta, onsite_n = -mu; the Kerr
 * extension adds onsite_nn1 = -U/2.  Any coefficient array may be NULL (zero).
 * pair must be zero in a Bose-Hubbard sector. */
typedef struct {
    int kind;      /* CVQ_BH or CVQ_BKC */
    int L;         /* modes */
    int N;         /* BH: total boson number */
    int d;         /* BKC: per-mode cutoff (even) */
    int parity;    /* BKC: 0 even sector, 1 odd sector */
    int periodic;  /* 1: bond (L-1, 0) present */
    const double *hop, *pair, *onsite_nn1, *onsite_n2, *onsite_n;  /* host arrays */
} cvq_model;

typedef struct cvq_sector cvq_sector;
typedef struct cvq_pool cvq_pool;

/* Message of the last error returned on this thread ("" if none). */
const char *cvq_last_error(void);

/* Build the sector indexer and Hamiltonian tables (Sec. III) on the current
 * device.  Copies everything it needs from *m.  Synchronises.  Errors:
 * EINVAL (limits, odd d, pair terms in BH), ENOMEM, ECUDA. */
int cvq_init_sector(const cvq_model *m, cvq_sector **out);
int cvq_sector_dim(const cvq_sector *s, int64_t *dim);
/* Host-side rank of the occupation tuple occ[0..L-1]; EINVAL if not in the sector. */
int cvq_sector_index(const cvq_sector *s, const int *occ, int64_t *index);
void cvq_destroy_sector(cvq_sector *s);

/* Build the operator pool (Sec. IV.B, Table I): for every generator its
 * block structure within the sector and the eigendecomposition of each
 * Hermitian block (host FP64 Jacobi), uploaded once.  ops is a host array of
 * K entries, copied.  Errors: EINVAL (bad type / modes / op that breaks the
 * sector symmetry), ENOMEM, ECUDA. */
int cvq_set_pool(const cvq_sector *s, const cvq_op *ops, int K, cvq_pool **out);
void cvq_destroy_pool(cvq_pool *p);

/* Device workspace, in bytes, needed by the calls below for ansatz length up
 * to n_max (and for screening the whole pool; p may be NULL for cvq_apply_H
 * alone).  Every call below takes (workspace, workspace_bytes): a caller-owned
 * device buffer of at least the size this returns for the call's n, which the
 * call uses as scratch (no allocation happens inside the calls).  EINVAL if
 * workspace_bytes is too small.  Calls that share one workspace must be
 * ordered (same stream). */
int cvq_workspace_bytes(const cvq_sector *s, const cvq_pool *p, int n_max, size_t *bytes);

/* sigma = H psi (matrix-free sector matvec), and if energy_dev != NULL also
 * *energy_dev = Re <psi|H|psi> (Sec. IV.A/B energy).  psi and sigma: dim
 * amplitudes, must not alias.  workspace: >= cvq_workspace_bytes(s, NULL, 0). */
int cvq_apply_H(const cvq_sector *s, const cvq_c128 *psi, cvq_c128 *sigma, double *energy_dev,
                void *workspace, size_t workspace_bytes, void *stream);

/* Pool screen, Eq. (grad): grad_dev[k] = <psi|[H, A_{ops[k]}]|psi> = 2 Re <H psi|A psi>
 * for every pool element (subset == NULL, n_subset ignored, K outputs) or for
 * the n_subset pool indices in the host array subset (n_subset outputs). */
int cvq_screen_pool(const cvq_sector *s, const cvq_pool *p, const cvq_c128 *psi, const int *subset,
                    int n_subset, double *grad_dev, void *workspace, size_t workspace_bytes, void *stream);

/* psi_out = exp(theta_n A_n) ... exp(theta_1 A_1) psi0 (Sec. IV.B ansatz),
 * A_k = pool element op_ids[k] (host ints), theta host doubles, n >= 0.
 * psi0 and psi_out may alias. */
int cvq_apply_ansatz(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta, int n,
                     const cvq_c128 *psi0, cvq_c128 *psi_out, void *workspace, size_t workspace_bytes,
                     void *stream);

/* E(theta) = <psi_n|H|psi_n> and its gradient dE/dtheta_k, k = 0..n-1, by a
 * reverse (adjoint) state sweep: lambda = H psi_n, then for k = n..1
 * g_k = 2 Re <lambda|A_k psi_k>, psi <- U_k^dag psi, lambda <- U_k^dag lambda.
 * E_dev: 1 double, grad_dev: n doubles (device).  psi0 is not modified. */
int cvq_energy_and_grad(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta, int n,
                        const cvq_c128 *psi0, double *E_dev, double *grad_dev, void *workspace,
                        size_t workspace_bytes, void *stream);

/* cvq_energy_and_grad with checkpointed forward states, for large sectors
 * and deep ansatze: during the forward sweep psi is stored before the first
 * segment (a block gate or a run of diagonal gates) whose first gate index
 * reaches every, 2 every, ...; the reverse sweep replaces its recomputed psi
 * by the stored copy at each of those points, so rounding drift of
 * psi <- U^dag psi is bounded by `every` gates.  ckpt: device buffer of at
 * least cvq_checkpoint_bytes(s, n, every) bytes, 256-byte aligned (may be
 * NULL when that is 0).  Errors as cvq_energy_and_grad, plus EINVAL for
 * every < 1 or a short checkpoint buffer. */
int cvq_checkpoint_bytes(const cvq_sector *s, int n, int every, size_t *bytes);
int cvq_energy_and_grad_ckpt(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta, int n,
                             const cvq_c128 *psi0, double *E_dev, double *grad_dev, int every, void *ckpt,
                             size_t ckpt_bytes, void *workspace, size_t workspace_bytes, void *stream);

/* cvq_energy_and_grad with the forward states kept instead of recomputed
 * (Sec. IV.B adjoint gradient, the same E and g): during the forward sweep
 * each segment (a block gate, or a run of diagonal gates) leaves what the
 * reverse sweep needs of psi at its output in `states`: the amplitudes a
 * block gate changes, in the order of its tile table (blocks of one member
 * are unchanged and have no gradient term), or the whole df state after a
 * run of diagonal gates or an untiled block gate.  The reverse sweep then
 * forms each gradient term from the stored psi and updates only lambda, so
 * it reads and writes half the state traffic and does half the block
 * arithmetic of cvq_energy_and_grad, in exchange for device memory.
 *   cvq_stored_states_bytes: size of `states` for this ansatz (host op ids);
 *     it depends on which operators are block gates and on their tables.
 *   cvq_energy_and_grad_stored: states is a device buffer of at least that
 *     many bytes, 256-byte aligned (may be NULL when the size is 0), owned by
 *     the caller and overwritten.  Errors as cvq_energy_and_grad, plus
 *     EINVAL for a short or misaligned buffer or a projected pool. */
int cvq_stored_states_bytes(const cvq_sector *s, const cvq_pool *p, const int *op_ids, int n, size_t *bytes);
int cvq_energy_and_grad_stored(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta, int n,
                               const cvq_c128 *psi0, double *E_dev, double *grad_dev, void *states,
                               size_t states_bytes, void *workspace, size_t workspace_bytes, void *stream);

/* Projected gates (Sec. V.A): each gate's matrix elements are those of the
 * untruncated gate between states inside the cutoff, and the state is
 * renormalised after every gate that the cutoff makes non-unitary (the block
 * gates of a Kitaev-chain sector; diagonal gates stay unitary).  The
 * untruncated elements are obtained from each block's chain extended to the
 * inner cutoff: exact for beam splitters once inner_cutoff >= 2d - 1,
 * converging with inner_cutoff for squeezers.
 *   cvq_set_pool_projected: as cvq_set_pool, on a Kitaev-chain sector, with
 *     d <= inner_cutoff <= 64 (EINVAL otherwise).  Such a pool works with
 *     cvq_screen_pool (at theta = 0 the projected and truncated generators
 *     agree) and with the calls below; cvq_apply_ansatz and
 *     cvq_energy_and_grad reject it.
 *   cvq_projected_states_bytes: size of the caller's state buffer for an
 *     ansatz: one state per segment boundary (block gate or run of diagonal
 *     gates) plus the theta derivatives of the block unitaries.
 *   cvq_apply_ansatz_projected: the normalised psi_n.
 *   cvq_energy_and_grad_projected: E = <psi_n|H|psi_n> and dE/dtheta through
 *     the normalisations: with lambda = H psi_n, for each block gate
 *     mu = (lambda - Re<psi_k|lambda> psi_k) / N_k, g_k = 2 Re<mu|D_k psi_{k-1}>,
 *     lambda <- U_k^dag mu (every psi_k is kept in the state buffer).
 * states: device, 256-byte aligned, >= cvq_projected_states_bytes; workspace as
 * for cvq_energy_and_grad.  Errors: EINVAL, ENOMEM, ECUDA. */
int cvq_set_pool_projected(const cvq_sector *s, const cvq_op *ops, int K, int inner_cutoff, cvq_pool **out);
int cvq_projected_states_bytes(const cvq_sector *s, const cvq_pool *p, const int *op_ids, int n, size_t *bytes);
int cvq_apply_ansatz_projected(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta, int n,
                               const cvq_c128 *psi0, cvq_c128 *psi_out, void *states, size_t states_bytes,
                               void *workspace, size_t workspace_bytes, void *stream);
int cvq_energy_and_grad_projected(const cvq_sector *s, const cvq_pool *p, const int *op_ids, const double *theta,
                                  int n, const cvq_c128 *psi0, double *E_dev, double *grad_dev, void *states,
                                  size_t states_bytes, void *workspace, size_t workspace_bytes, void *stream);

/* One step of the Lanczos recurrence used for the exact ground energy E0
 * that defines Delta E = |E - E0| (Sec. IV.B stopping rule; exact
 * diagonalisation there).  Before the call the caller has w = H v and
 * alpha_dev[0] = Re <v|H v> (cvq_apply_H with energy_dev = alpha_dev), v of
 * unit norm, and beta_prev_dev[0] = beta_{j-1} (0 for j = 0; v_prev then
 * ignored).  The call forms w <- w - alpha v - beta_{j-1} v_prev,
 * beta_dev[0] = ||w|| and v_next = w / ||w|| (v_next = w if ||w|| = 0).
 * v_next may alias v_prev; all vectors are dim amplitudes on the device.
 * workspace: >= cvq_workspace_bytes(s, NULL, 0). */
int cvq_lanczos_step(const cvq_sector *s, const cvq_c128 *v_prev, const cvq_c128 *v, cvq_c128 *w, cvq_c128 *v_next,
                     const double *alpha_dev, const double *beta_prev_dev, double *beta_dev, void *workspace,
                     size_t workspace_bytes, void *stream);

/* Algorithmic cost of one application of pool element `op` on the whole
 * sector: bytes (amplitudes read + written, 16 B each) and flops (a complex
 * multiply-add counts 8) of the forward gate and of its reverse step in
 * cvq_energy_and_grad (gradient term + U^dag on psi and lambda).  Blocks of
 * one member (zero generator: the gate is the identity there) are not
 * counted; the kernels skip them.  Host only. */
int cvq_op_cost(const cvq_sector *s, const cvq_pool *p, int op, double *fwd_bytes, double *fwd_flops,
                double *adj_bytes, double *adj_flops);

/* State features for the learned proposal (ranking pool operators before the
 * exact Eq. (grad) screen; the learned proposal extends Sec. IV.B): for the
 * state psi (dim amplitudes, device, not necessarily normalised) writes
 *   out_dev[r]               = <psi| n_r |psi>,          r = 0..L-1
 *   out_dev[L + r]           = <psi| n_r^2 |psi>,
 *   out_dev[2L + 2p], [+1]   = Re, Im <psi| a_i^dag a_j |psi>, (i, j) = (pair_i[p], pair_j[p]),
 * p = 0..npairs-1 (host arrays, i != j, 0 <= npairs <= 240).  The truncated
 * ladder rules of Sec. II.A apply.  workspace: >= cvq_features_workspace_bytes.
 * Errors: EINVAL, ECUDA. */
int cvq_features_workspace_bytes(const cvq_sector *s, int npairs, size_t *bytes);
int cvq_features(const cvq_sector *s, const cvq_c128 *psi, const int *pair_i, const int *pair_j, int npairs,
                 double *out_dev, void *workspace, size_t workspace_bytes, void *stream);

/* Learned proposal scorer (extends Sec. IV.B's operator selection): an MLP
 * that maps one pool operator's input features (in_dim = 32 floats) to a
 * score, 32 -> 256 -> 256 -> 1 with ReLU.  Weights are kept as fp32 master
 * copies and used as bf16 (round to nearest even) in every product; all sums
 * accumulate in fp32.  The parameter vector (74,497 floats) is laid out as
 * W1[256][32], b1[256], W2[256][256], b2[256], w3[256], b3.
 *   cvq_mlp_create: He-initialised weights from `seed`, room for max_rows rows
 *     (allocates; synchronises).
 *   cvq_mlp_forward: scores_dev[r] for the rows of X_dev (row-major, rows x 32,
 *     device); keeps the activations for cvq_mlp_backward.
 *   cvq_mlp_backward: gradients of sum_r dscores_dev[r] * score_r with respect
 *     to every parameter (overwrites the gradient buffer), for the rows of the
 *     last forward call.
 *   cvq_mlp_listwise_loss: for nlists lists (device offsets
 *     list_off_dev[0..nlists], rows list_off[l]..list_off[l+1]) of scores and
 *     target probabilities, loss_dev[l] = -sum p log softmax(s) and
 *     dscores_dev = softmax(s) - p; an empty list gives loss 0.  No
 *     allocation, no synchronisation.
 *   cvq_mlp_adam_step: one Adam step (lr, beta1 = 0.9, beta2 = 0.999,
 *     eps = 1e-8, bias-corrected for step t >= 1) on the master weights, then
 *     refreshes the bf16 copies.
 *   cvq_mlp_get / cvq_mlp_set: copy parameters (or, get only, gradients with
 *     which = 1) between the model and a host float array of 74,497 entries;
 *     set also zeroes the Adam moments and refreshes the bf16 copies.  Both
 *     synchronise the device.
 * Forward, backward and Adam run on `stream` without allocating or
 * synchronising; one model must not be used from two streams at once.
 * Errors: EINVAL (sizes), ENOMEM, ECUDA. */
typedef struct cvq_mlp cvq_mlp;
int cvq_mlp_create(int in_dim, int hidden, int max_rows, uint64_t seed, cvq_mlp **out);
void cvq_mlp_destroy(cvq_mlp *m);
int cvq_mlp_forward(cvq_mlp *m, const float *X_dev, int rows, float *scores_dev, void *stream);
int cvq_mlp_backward(cvq_mlp *m, const float *X_dev, int rows, const float *dscores_dev, void *stream);
int cvq_mlp_listwise_loss(const float *scores_dev, const float *targets_dev, const int *list_off_dev, int nlists,
                          float *dscores_dev, float *loss_dev, void *stream);
int cvq_mlp_adam_step(cvq_mlp *m, float lr, int t, void *stream);
int cvq_mlp_get(const cvq_mlp *m, int which, float *host, size_t n);
int cvq_mlp_set(cvq_mlp *m, const float *host, size_t n);

/* Batched engine (extends Sec. IV.B's per-instance evaluation to many
 * Hamiltonian instances at once, e.g. a U/J sweep): the energy and adjoint
 * gradient of every instance of the batch from one CUDA graph launch.
 *   cvq_batch_create: n_inst sectors of one kind on the current device, each
 *     with its pool (pools[i] built on sectors[i]); room for n_max gates per
 *     instance.  Allocates 32 bytes per amplitude per instance plus the block
 *     unitaries.  The sectors and pools must outlive the batch.
 *   cvq_batch_set_ansatz: the ansatz of every instance, n_ops[i] in [-1,
 *     n_max] (-1: instance left out), op ids packed instance after instance
 *     (host), psi0[i] the device complex128 reference state of instance i
 *     (kept by pointer).  Builds the work schedule (allocates, synchronises).
 *   cvq_batch_set_schedule: work-item size in amplitudes (tile >= 256) and
 *     CTAs per SM of every layer launch (1 or 2); rebuilds the schedule.
 *   cvq_batch_energy_and_grad: theta_dev and grad_dev packed like the op ids,
 *     E_dev[i] per instance (device, float64); instances left out are not
 *     written.  The first call for a schedule (or for new buffer pointers)
 *     captures the evaluation into a CUDA graph; later calls launch it on
 *     `stream`.  Results are deterministic: every partial sum has its own
 *     slot and the final sums run in a fixed order.
 *   cvq_batch_set_active: active[i] = 0 pauses instance i (its items are
 *     skipped and its outputs not written) without a new schedule or graph;
 *     set_ansatz makes every instance with an ansatz active.  Synchronises
 *     `stream`.
 *   cvq_batch_info: kernels per evaluation, work items, layers and the
 *     number of parameters.
 * Errors: EINVAL (sizes, mixed kinds or devices, op ids), ENOMEM, ECUDA. */
typedef struct cvq_batch cvq_batch;
int cvq_batch_create(const cvq_sector *const *sectors, const cvq_pool *const *pools, int n_inst, int n_max,
                     cvq_batch **out);
void cvq_batch_destroy(cvq_batch *b);
int cvq_batch_set_ansatz(cvq_batch *b, const int *n_ops, const int *op_ids, const cvq_c128 *const *psi0);
int cvq_batch_set_schedule(cvq_batch *b, int64_t tile, int ctas_per_sm);
int cvq_batch_energy_and_grad(cvq_batch *b, const double *theta_dev, double *E_dev, double *grad_dev, void *stream);
int cvq_batch_set_active(cvq_batch *b, const int *active, void *stream);
int cvq_batch_info(const cvq_batch *b, int *kernels_per_eval, int *items, int *layers, int64_t *n_params);

/* Batched pool screen, Eq. (grad) (the selection step of Sec. IV.B for every
 * instance of the batch at once): for every active instance i with an
 * ansatz, psi_i = U_i(theta_i) psi0_i is formed from the instance's ansatz
 * (cvq_batch_set_ansatz) at theta_dev (packed like the op ids), and
 *   grad_dev[o_i + k] = <psi_i|[H_i, A_{s_i[k]}]|psi_i>
 * for the pool indices s_i: every pool element 0..K_i-1 when subset_off is
 * NULL, else subset[subset_off[i] .. subset_off[i+1]) (host arrays;
 * subset_off has n_inst + 1 nondecreasing entries from 0).  The outputs are
 * packed instance after instance: o_i is the number of outputs of the
 * instances before i, instances without an ansatz (n_ops = -1) having none.
 * Inactive instances (cvq_batch_set_active) are not written.  Per instance
 * the screen shares one neighbour read among all elements with the same
 * ladder shift, and every partial sum has its own slot, summed in a fixed
 * order: results are deterministic.  The first call for an ansatz structure,
 * schedule, subset list or pair of buffer pointers builds a plan (allocates,
 * synchronises) and captures it in a CUDA graph; later calls launch the
 * graph on `stream`.  Calls on one batch (screens and evaluations) must be
 * ordered: they share the batch's state buffers.  Errors: EINVAL (sizes,
 * indices outside a pool), ENOMEM, ECUDA. */
int cvq_batch_screen(cvq_batch *b, const double *theta_dev, const int *subset_off, const int *subset, double *grad_dev,
                     void *stream);

/* Pool screen for callers that cannot allocate device memory.  The paper has
 * no counterpart to this call.  It exists for code that must not call
 * cudaMalloc when it screens: latency-critical loops that cannot pay for the
 * device-wide synchronisation an allocation brings, host applications whose
 * own caching allocator has reserved all of the device's memory (so an
 * allocation by this library would fail), and plug-ins that their host hands
 * fixed buffers and forbids allocating.  It computes the same values as
 * cvq_screen_pool for the n_subset pool indices in the host array subset
 * (1 <= n_subset <= 64, EINVAL otherwise) and writes them to
 * grad_dev[0..n_subset), with no workspace: psi is read as complex128, and
 * each row of H psi is formed on the fly, once per pass over the sector for
 * every 8 screened elements (a call costs about ceil(n_subset / 8)
 * matvecs, against one pass per 8 distinct ladder shifts for
 * cvq_screen_pool).  The per-block partial sums live in a fixed device array
 * of 64 x 608 doubles (311,296 bytes) that every GPU which loads the library
 * keeps until the process exits.  The first call on a device (and the first
 * after a device reset, which gives the array a new address) looks up that
 * array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture.  All calls on a device share the array: calls
 * that overlap on the GPU (different streams without ordering) race and give
 * wrong results.  Each call overwrites the array rows it reads, so no
 * clearing is needed.  Errors: EINVAL, ECUDA. */
int cvq_screen_subset_noalloc(const cvq_sector *s, const cvq_pool *p, const cvq_c128 *psi, const int *subset,
                              int n_subset, double *grad_dev, void *stream);

/* Live per-kernel timing.  cvq_profile_start(capacity) makes every later
 * launch by this library (any thread, any stream) record a CUDA event pair on
 * its stream, up to `capacity` launches; cvq_profile_stop waits for those
 * events, writes one record per kernel kind into out[0..max_out) (*n_out of
 * them), and turns timing off.  Each record sums launches, device time and
 * the algorithmic bytes and flops of those launches.  Errors: EINVAL, ECUDA. */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;
    double bytes;
    double flops;
} cvq_kernel_stat;

int cvq_profile_start(int capacity);
/* Time only one launch in `every` of each kernel kind (default 1: all).  The
 * others are still counted (launches, bytes, flops), and a kind's device time
 * is its timed launches' time scaled to all of its launches; fewer event
 * records keep the host's launch path short.  Takes effect at the next
 * cvq_profile_start. */
int cvq_profile_sample(int every);
int cvq_profile_stop(cvq_kernel_stat *out, int max_out, int *n_out);

#ifdef __cplusplus
}
#endif
#endif /* CVQ_H */
