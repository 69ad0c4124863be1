/*
 * mld.h - C ABI of the GB300 (sm_103a) tensor-network maximum-likelihood
 * decoder for the rotated surface code under independent Pauli noise.
 *
 * Method (arxiv 2605.17230): for each syndrome s and logical class l the
 * coset partition function Z_l(s) = sum_{E in C_l(s)} Pr(E) (Eq. 3, Sec. 2.3)
 * is computed in the generator picture (Eq. 7, Sec. 3.2.1) by a boundary-MPS
 * sweep over the corner columns of the patch, compressed to bond dimension
 * chi after every column; the decision is argmax_l Z_l(s) (Eq. 4).
 *
 * Conventions (the paper's lattice figure is not available; this is the
 * layout adopted, exported by mld_code_layout):
 *  - d odd, 3 <= d <= 25; n = d*d data qubits, qubit (r,c) has index r*d+c.
 *  - Plaquette (i,j), 0 <= i,j <= d, acts on qubits (i-1,j-1),(i-1,j),(i,j-1),
 *    (i,j) inside the patch; it is X-type if i+j is even, Z-type if odd.
 *    Interior plaquettes are all checks; rows 0 and d keep only the X-type
 *    weight-2 ones, columns 0 and d only the Z-type weight-2 ones: n-1 checks.
 *  - Stabiliser index = column-major order (j outer, i inner) of the checks.
 *    Syndrome bit k lives in word k/64, bit k%64 of a uint64 row of
 *    syn_words = ceil((n-1)/64) words.
 *  - Logical operators: Z_L = Z on row 0, X_L = X on column 0. The class of
 *    an error E is l = l_X + 2 l_Z with l_X = <E,Z_L>, l_Z = <E,X_L>, i.e. the
 *    output order is I, X, Z, Y.
 *  - Noise (independent Pauli noise, Sec. 3.1.1): float rows
 *    (p_I, p_X, p_Y, p_Z) per qubit, or one depolarizing strength p per
 *    syndrome (p_I = 1-p, p_X = p_Y = p_Z = p/3, Sec. 2.2).
 *
 * Errors: every call returns an mld_status; nothing is thrown across the
 * ABI. Device-side failures (a Jacobi sweep that hits its iteration bound,
 * a non-finite value) are reported through a library-owned status word that
 * is read when the call synchronises (mld_decode_host, or
 * mld_decode_status after the caller has synchronised the stream).
 */
#ifndef MLD_H
#define MLD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mld_code mld_code;   /* opaque, owned by the library */

typedef enum {
    MLD_OK = 0,
    MLD_ERR_INVALID_ARG = 1,   /* bad d, chi < 1, B < 0, NULL pointer, bad mode */
    MLD_ERR_UNSUPPORTED = 2,   /* valid request this build cannot run (e.g. too
                                  much on-chip memory for this d and chi) */
    MLD_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    MLD_ERR_NOMEM = 4,         /* device or host allocation failed */
    MLD_ERR_TIMEOUT = 5,       /* a bounded device loop hit its limit */
    MLD_ERR_NUMERIC = 6        /* a non-finite value appeared on the device */
} mld_status;

typedef enum {
    MLD_FP32 = 0,              /* FP32 storage and arithmetic, FP32 Jacobi
                                  rotations; FP64 only where ln Z is formed
                                  from the mantissa and the power-of-two
                                  exponent */
    MLD_MIXED_BF16 = 1,        /* reserved: MLD_ERR_UNSUPPORTED (BF16 operands
                                  miss |d ln Z| <= 1e-3 on the leading coset) */
    MLD_MIXED_TF32 = 2,        /* data-site MPO.MPS products on the tensor
                                  cores from operands split into two TF32
                                  parts (hi.hi + hi.lo + lo.hi), FP32
                                  accumulate; untruncated chi only. The split
                                  products run at d = 9 and 11, where they are
                                  faster; at other d the FP32 products run
                                  (same or better accuracy) */
    MLD_FP64 = 3               /* complex FP64 elimination; mld_decode_xz
                                  only (other entry points return
                                  MLD_ERR_INVALID_ARG) */
} mld_precision;

typedef enum {
    MLD_NOISE_TABLE = 0,       /* noise = float[n][4] shared by the batch */
    MLD_NOISE_DEPOL = 1        /* noise = float[B], depolarizing p per syndrome */
} mld_noise_mode;

/* Build the rotated distance-d code: check supports, logical operators and a
 * destabiliser table (for each check k a Pauli T_k that anticommutes with
 * check k only and commutes with X_L and Z_L), from which the pure error of
 * a syndrome, f(s) = prod_{s_k=1} T_k, is formed (Sec. 3.2.1, the fixed
 * representative E_{l,s}). Host-only: device copies are made by the first
 * decode call. *out is owned by the caller and released with
 * mld_code_destroy. MLD_ERR_INVALID_ARG unless d is odd and 3 <= d <= 25. */
mld_status mld_code_create_rotated(int d, mld_code** out);

/* Host-side pure errors: reps[B][4][n] receives the Pauli codes (x + 2z) of
 * the representatives E_{l,s} = f(s) * X_L^{l_X} * Z_L^{l_Z}, l = I, X, Z, Y,
 * for B host syndromes (Sec. 3.2.1: the fixed representative whose coset the
 * generator-picture sum runs over). Needs no GPU. */
mld_status mld_code_representatives(const mld_code* code, const uint64_t* syndromes, int64_t B,
                                    uint8_t* reps);

/* Release a code and every device buffer it owns. NULL is allowed. */
void mld_code_destroy(mld_code* code);

/* n_qubits = d*d, n_stabs = d*d-1, syn_words = ceil(n_stabs/64). Any output
 * pointer may be NULL. */
mld_status mld_code_info(const mld_code* code, int* n_qubits, int* n_stabs, int* syn_words);

/* Host arrays: stab_type[n_stabs] (0 = X-type, 1 = Z-type),
 * stab_qubits[n_stabs][4] (qubit indices, -1 padded), logical_x[n] (1 on the
 * support of X_L), logical_z[n] (1 on the support of Z_L). Any may be NULL. */
mld_status mld_code_layout(const mld_code* code, int32_t* stab_type, int32_t* stab_qubits,
                           uint8_t* logical_x, uint8_t* logical_z);

/* Decode B syndromes on the GPU (Eq. 3, 4 and 7; boundary MPS of Sec. 3.2.1).
 *   noise      device pointer: float[n][4] (MLD_NOISE_TABLE) or float[B]
 *              (MLD_NOISE_DEPOL). Rows are (p_I, p_X, p_Y, p_Z).
 *   syndromes  device pointer, uint64[B][syn_words].
 *   chi        maximum bond dimension kept after each column (chi >= 1).
 *              chi >= 2^floor(d/2) discards nothing: the result is then the
 *              exact ln Z_l(s) up to rounding. Below that it is the
 *              boundary-MPS approximation for the representative
 *              f(s) * X^{l_X} * Z_L^{l_Z} with X^{l_X} the X string on column
 *              d-1 (an X_L of the same cosets; the two classes l_X = 0, 1
 *              then share every column but the last, which the kernels sweep
 *              once and reuse).
 *   precision  an mld_precision value.
 *   logP       device pointer, double[B][4]: ln Z_l(s) for l = I, X, Z, Y
 *              (the joint log-probability ln Pr(s, l); ln Pr(l|s) is
 *              logP - logsumexp(logP), Eq. 3). -inf when Z_l(s) = 0.
 *   argmax     device pointer uint8[B] or NULL: argmax_l Z_l(s), ties and
 *              all--inf rows go to the lowest class index.
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Which kernel runs: see mld_code_set_exact_kernel (untruncated chi; the
 * same exact boundary state held as MPS sites or, at d = 11 and 13 by
 * default, densely) and mld_code_set_truncation_kernel (truncating chi).
 * All arrays are caller-owned device memory; the call is asynchronous and
 * allocates nothing per call once a call for the same (code, chi) and at
 * least the same B has been made (the first uploads the column plan and
 * sizes the workspaces). Status of the device work: see
 * mld_decode_status; a noise row that is not a probability distribution
 * (an entry negative or non-finite, or the row's sum off 1 by more than
 * 1e-6) or a depolarizing strength outside [0, 1] is reported there as
 * MLD_ERR_INVALID_ARG (checked on the device before the decode, so the call
 * itself stays asynchronous). B = 0 is a no-op. */
mld_status mld_decode(const mld_code* code, const float* noise, int noise_mode,
                      const uint64_t* syndromes, int64_t B, int chi, int precision,
                      double* logP, uint8_t* argmax, void* stream);

/* The same with HOST pointers: copies the inputs to the device, decodes,
 * copies the results back and synchronises. Device buffers are cached in the
 * code object and grown on demand. argmax may be NULL. */
mld_status mld_decode_host(const mld_code* code, const float* noise, int noise_mode,
                           const uint64_t* syndromes, int64_t B, int chi, int precision,
                           double* logP, uint8_t* argmax);

/* mld_decode without any device allocation, for callers that cannot
 * allocate device memory (a real-time loop that must not stall on the
 * device-wide synchronisation of cudaMalloc, or a process whose device memory
 * is already reserved by another framework's caching allocator). The paper
 * has no counterpart: this is a deployment variant of the untruncated sweep.
 *   Scope: precision MLD_FP32, chi at or above the exact bond of every cut
 *   (no truncation), and 3 <= d <= 11; anything else returns
 *   MLD_ERR_UNSUPPORTED.
 *   Scratch: the status word and the code's destabiliser tables live in one
 *   16 KiB file-scope __device__ array that every GPU loading the library
 *   holds until the process exits; a code whose tables do not fit returns
 *   MLD_ERR_UNSUPPORTED. Each call resets the status word; the tables are
 *   copied (asynchronously on `stream`, from pageable host memory) only when
 *   the array holds another code's tables. The array keeps the last call's
 *   contents, so calls that overlap on the GPU (other streams, other
 *   threads) race and must be serialised by the caller.
 *   Set-up: the first call on a device looks up the array's device address
 *   (the device must be current); make that first call before any stream
 *   capture.
 *   Arguments as mld_decode. check_status != 0 synchronises the stream and
 *   returns the device status (MLD_OK, MLD_ERR_INVALID_ARG for invalid noise
 *   values as in mld_decode, MLD_ERR_NUMERIC or MLD_ERR_TIMEOUT); 0 returns as
 *   soon as the work is enqueued, and the device status of that call cannot
 *   be read afterwards (mld_decode_status reads another word, and the next
 *   call clears this one). */
mld_status mld_decode_noalloc(const mld_code* code, const float* noise, int noise_mode,
                              const uint64_t* syndromes, int64_t B, int chi, int precision,
                              double* logP, uint8_t* argmax, void* stream, int check_status);

/* One decode job of a mixed batch: arguments of mld_decode (device pointers). */
typedef struct {
    const mld_code* code;
    const float* noise;
    int noise_mode;
    const uint64_t* syndromes;
    int64_t B;
    int chi;
    int precision;
    double* logP;
    uint8_t* argmax;             /* may be NULL */
} mld_job;

/* Decode a batch of jobs of different d, noise and chi (the batching of
 * independent syndromes across codes; the paper has no counterpart). Jobs run
 * concurrently on library-owned streams forked from `stream` and joined back
 * into it; jobs that share a code object run one after another (they share
 * its workspace). Asynchronous; statuses as mld_decode. */
mld_status mld_decode_batch(const mld_job* jobs, int n_jobs, void* stream);

typedef struct mld_graph mld_graph;   /* opaque */

/* Capture mld_decode_batch(jobs) into an executable CUDA graph: one graph
 * launch then decodes every job again, on whatever the job buffers hold at
 * that time (the buffer pointers are fixed at capture). The jobs are run
 * once, uncaptured, before the capture so that every plan and workspace is
 * allocated (and every autotuned shape chosen) first. */
mld_status mld_graph_create(const mld_job* jobs, int n_jobs, mld_graph** out);
mld_status mld_graph_launch(mld_graph* graph, void* stream);
void mld_graph_destroy(mld_graph* graph);

/* Time the candidate CTA shapes (warps per block) of this code, chi and
 * precision on a synthetic batch of the given size and keep the fastest for
 * later decodes of this code object (per chi and precision). Where the
 * per-warp state exceeds a block's shared memory (d = 13 untruncated) the
 * candidates are the resident warps per SM of the global-workspace sweep
 * (2, 4, 8, 16; *chosen_warps reports that count). At an untruncated chi
 * with d = 9, 11 or 13 the dense-state kernel is a candidate too, and the faster
 * kernel is kept for that chi (*chosen_warps = 0 when it is the dense one),
 * unless mld_code_set_exact_kernel forces one. For a
 * truncating chi the rank-adaptive sweep (4 units per block) is a candidate
 * beside the fixed-shape sweep's shapes, and the faster kernel is kept for
 * that chi (unless mld_code_set_truncation_kernel forces one). Synchronous. */
mld_status mld_autotune(const mld_code* code, int chi, int precision, int64_t sample_B, int* chosen_warps);

/* Adjoint of the sweep: derivatives of ln Z_l(s) with respect to the noise
 * table (Sec. 3.2.4: the contraction is differentiable in the local error
 * probabilities; Eq. 10's estimation back-propagates through it).
 *   noise      device float[n][4] (MLD_NOISE_TABLE only).
 *   dlogP      device double[B][4] upstream gradient dL/d ln Z_l(s), or NULL
 *              (then only logP is computed).
 *   logP       device double[B][4] output (ln Z_l(s)), or NULL.
 *   dnoise     device double[n][4]: dL/dp_{q,P} (all four entries of a row
 *              treated as independent) is ADDED to it.
 * Each qubit factor's environment is contracted exactly, so chi must not
 * truncate (MLD_ERR_UNSUPPORTED otherwise) and d <= 13. The left and right
 * boundary states are kept dense (the right states are carried back through
 * each column by the transposed factors): on chip for d <= 11; at d = 13 the
 * states inside a column (128 KB each) live in a device workspace of about
 * 1.7 MB per resident block, the corner-column states on chip. The left
 * state at every column boundary is stored by the forward pass (a
 * checkpoint per column) and the states inside a column are recomputed from
 * it during the backward pass. FP32 contraction, FP64
 * accumulation in a fixed order, so reruns give the same bits. Asynchronous
 * on stream; uses a device workspace owned by the code object (not reentrant
 * per code). */
mld_status mld_decode_grad(const mld_code* code, const float* noise, const uint64_t* syndromes, int64_t B,
                           int chi, const double* dlogP, double* logP, double* dnoise, void* stream);

/* Read and clear the device status word written by earlier mld_decode and
 * mld_decode_grad calls on this code (the caller must have synchronised
 * their streams): MLD_OK, MLD_ERR_INVALID_ARG (invalid noise values),
 * MLD_ERR_NUMERIC or MLD_ERR_TIMEOUT, in that order of precedence. */
mld_status mld_decode_status(const mld_code* code);

/* Relative cutoff of the truncating SVDs (Sec. 3.2.1 discards the smallest
 * singular values; this sets which of them count as resolved). At every cut
 * of a truncating chi the compression keeps the k largest singular values,
 * k = min(chi, #{sigma_j > rel * sigma_1}). Default 1e-7: values below it lie
 * under the FP32 resolution of the bond matrix, and dropping them lets the
 * kernel run on the numerical rank of each cut (6..27 at p = 0.12, d = 17
 * and 25) instead of chi. rel = 0 keeps min(chi, number of values) exactly.
 * Applies to later decodes of this code object. MLD_ERR_INVALID_ARG unless
 * 0 <= rel < 1. Host only. */
mld_status mld_code_set_svd_cutoff(mld_code* code, double rel);

/* Which kernel decodes a truncating chi for this code: 0 (default) per chi,
 * mld_autotune's choice if it timed this chi, else the fixed-shape sweep when
 * its whole per-warp state fits 24 KB of shared memory (small d and chi) and
 * the rank-adaptive sweep otherwise; 1 always the rank-adaptive sweep (one
 * warp per (syndrome, l_Z), runtime bonds, pivoted QR, Jacobi on R^T); 2
 * always the fixed-shape sweep (one warp per unit, every bond at its
 * chi-capped size, values below the cutoff written as zero). Both apply the
 * same truncation rule. MLD_ERR_INVALID_ARG for other values. Host only. */
mld_status mld_code_set_truncation_kernel(mld_code* code, int which);

/* Largest bond capacity of the rank-adaptive sweep's first pass, which runs
 * on every resident warp with a global slice per warp: 48 (2.25 MB a warp),
 * 64 (4.5 MB) or 128 (17.8 MB; 45 GB on 152 SMs x 16 warps); 0 (default)
 * the smallest of these that holds chi. Units whose bonds exceed the first
 * pass's capacity restart in a second pass on few warps, a serial tail; a
 * lower cap trades that tail for workspace. If a workspace cannot be
 * allocated the next smaller capacities are used. MLD_ERR_INVALID_ARG for
 * other values. Applies to later decodes of this code. Host only. */
mld_status mld_code_set_truncation_workspace(mld_code* code, int max_bond);

/* Which kernel decodes an untruncated chi (chi >= 2^floor(d/2), where the
 * boundary MPS of Sec. 3.2.1 discards nothing and is the exact boundary state
 * over one corner column): 0 (default) mld_autotune's choice for that chi if
 * it timed one, else the dense-state kernel at d = 11 and 13 (the faster
 * one there) and the boundary-MPS kernel elsewhere; 1 always the
 * boundary-MPS kernel (sites at the exact cut ranks, compile-time plan per
 * d; split-TF32 tensor-core products for MLD_MIXED_TF32 at d = 9, 11); 2
 * the dense-state kernel (d = 9, 11, 13: one block per (syndrome, l_Z) keeps
 * the 2^(d+2)-entry state of a column in shared memory and applies the
 * qubit factors to it in place; FP32 for either precision). Both give ln Z_l
 * to FP32 accuracy. MLD_ERR_INVALID_ARG for other values,
 * MLD_ERR_UNSUPPORTED for 2 at other d. Host only. */
mld_status mld_code_set_exact_kernel(mld_code* code, int which);

/* Floating-point operations executed by the truncating sweeps of this code
 * since the last call (apply, QR, Q applications and every Jacobi pair
 * evaluation and rotation actually performed, counted on the device), then
 * reset to zero. The caller synchronises the decode streams first. Untruncated
 * decodes are not counted here (see mld_decode_flops). */
mld_status mld_decode_executed_flops(const mld_code* code, double* flops);

/* Histogram of the bonds kept at the truncating cuts of this code's decodes
 * since the last call: hist[k] (k = 1..63) counts cuts that kept k singular
 * values, hist[64] those that kept 64 or more; hist[0] counts site steps
 * whose buffers did not fit the on-chip arena and ran in the global spill
 * arena (rank-adaptive kernel only); then reset. The caller synchronises the
 * decode streams first. */
mld_status mld_decode_bond_histogram(const mld_code* code, int64_t* hist /* [65] */);

/* Counted floating-point operations per syndrome (all four classes) of the
 * sweep schedule that mld_decode runs for this code, chi and precision: the
 * MPO.MPS products, the QR and Q applications of truncating columns and the
 * bond-matrix products, from the same shape plan the kernel executes
 * (columns 0..d-2 are swept once per l_Z and shared by l_X = 0, 1, whose
 * representatives differ only in the last column). Jacobi
 * SVD work, which depends on the data, is not included. Host only. */
mld_status mld_decode_flops(const mld_code* code, int chi, int precision, double* flops_per_syndrome);

/* Detector-picture MLD of a code-capacity detector error model (Sec. 3.2.2:
 * the network of error-mechanism tensors diag(1-p, p), one parity tensor
 * delta(XOR of incident bits = s_j) per detector and the logical parity
 * tensors, contracted without reference to a stabiliser coset).
 * The model is n_mech independent mechanisms; mechanism m applies Pauli
 * mech_pauli[m] (code x + 2z: 1 = X, 2 = Z, 3 = Y) to qubit mech_qubit[m]
 * (index r*d + c) with probability mech_p[m]. These three are HOST arrays,
 * read before the call returns. Z_l(s) sums the probability of every
 * mechanism configuration whose syndrome is s and whose logical parities
 * (x-parity on Z_L's support, row 0; z-parity on X_L's support, column 0)
 * equal those of the class-l representative, l = l_X + 2 l_Z as in
 * mld_decode; the result equals mld_decode with each qubit's table the
 * distribution of the product of its mechanisms.
 *   syndromes  device uint64[B][words]
 *   logP       device double[B][4]: ln Z_l(s) (-inf for an impossible class)
 *   argmax     device uint8[B] or NULL (ties -> lowest class)
 * The contraction is exact: one thread block per syndrome keeps the dense
 * boundary state over the open detectors' partial parities and both
 * logical parities, all four classes in one sweep; FP32 with power-of-two
 * rescaling per column, ln Z in FP64. d <= 11 (the state at d = 11 is
 * 2^15 floats, one block of 512 threads per SM; MLD_ERR_UNSUPPORTED
 * otherwise); MLD_ERR_INVALID_ARG for a mechanism with a qubit outside
 * [0, n), a code outside 1..3 or p outside [0, 1]. Asynchronous on stream;
 * no device allocation. */
mld_status mld_decode_dem(const mld_code* code, const int32_t* mech_qubit, const int32_t* mech_pauli,
                          const double* mech_p, int32_t n_mech, const uint64_t* syndromes, int64_t B,
                          double* logP, uint8_t* argmax, void* stream);

/* MLD under independent X/Z noise by Kac-Ward determinants (Sec. 3.1.3:
 * the planar random-bond Ising model of each part, Z proportional to
 * sqrt(det(I - Lambda)) per logical sector). Qubit q flips its X part with
 * probability px[q] and its Z part with probability pz[q], independently:
 * Pr(E) = prod_q px^x (1-px)^(1-x) pz^z (1-pz)^(1-z), so the class
 * probabilities factorise, Z_l = ZX_{l_X} ZZ_{l_Z}. Classes and their order
 * are those of mld_decode (l = l_X + 2 l_Z); the result equals mld_decode with
 * the table (1-px)(1-pz), px(1-pz), px pz, (1-px) pz (I, X, Y, Z).
 *   px         device float[n], each in (0, 1)
 *   pz         device float[n], each in (0, 1); NULL for bit-flip noise (no Z
 *              errors): ln Z is -inf for l_Z = 1, and for every class of a
 *              syndrome whose X-type part is nonzero
 *   syndromes  device uint64[B][words]
 *   precision  MLD_FP32 or MLD_FP64 (complex arithmetic of that type)
 *   logP       device double[B][4]: ln Z_l(s)
 *   argmax     device uint8[B] or NULL (ties -> lowest class)
 * Exact in exact arithmetic at any odd d >= 3 up to 25. Each part is one
 * banded elimination with partial pivoting (order 2|E| = 2d^2 + O(d),
 * bandwidth 3d), one warp per syndrome up to d = 13 and one block of four
 * warps per syndrome above, the two sectors sharing all but a final 4 x 4
 * determinant. The determinant is a sum of signed terms, so accuracy
 * follows the conditioning of the matrix: a class far less likely than the
 * leading one carries an error of order eps * cond relative to the leading
 * class's Z, and at low error rates the leading class too. Measured against
 * MLD_FP64 (4,096 syndromes per point): MLD_FP32 keeps the leading ln Z
 * within 1.1e-3 at p = 0.10 up to d = 25, but on rare syndromes reaches
 * 0.097 (p = 0.05) and 0.29 (p = 0.02) at d = 25; one decision in 4,096
 * differed at d = 17, p = 0.02. Use MLD_FP64 for ln Z at low rates. A probability
 * outside (0, 1) sets MLD_ERR_INVALID_ARG in the status word
 * (mld_decode_status); a vanishing pivot sets MLD_ERR_NUMERIC and gives -inf.
 * The first call for a code builds the graph and copies it to the device
 * (synchronous, a few hundred KB); later calls are asynchronous on stream
 * with no allocation. MLD_ERR_UNSUPPORTED if a syndrome's window exceeds
 * the device's shared memory per block (it fits up to d = 25 in FP64 on
 * GB300: 200 KB). */
mld_status mld_decode_xz(const mld_code* code, const float* px, const float* pz, const uint64_t* syndromes,
                         int64_t B, int precision, double* logP, uint8_t* argmax, void* stream);

/* Floating-point operations executed by mld_decode_xz on this code since the
 * last call (per elimination step: a complex multiplier, 6 flops, and a
 * complex multiply-subtract, 8 flops, per updated column of every row with a
 * nonzero multiplier, counted on the device from the step's actual extent),
 * then reset to zero. The caller synchronises the decode streams first. */
mld_status mld_decode_xz_executed_flops(const mld_code* code, double* flops);

/* Measurement helper (not part of the method): times a kernel of independent
 * FP32 FMA chains on every SM of the current device for about `seconds` and
 * returns the sustained rate in TFLOP/s (2 flops per FMA) and the SM count,
 * the denominator of the FP32 sweep kernels' roofline. Synchronous; allocates
 * a small buffer. */
mld_status mld_measure_fp32_peak(double seconds, double* tflops, int* sm_count);

/* Number of kernel launches one mld_decode call with an argmax output makes
 * (the noise check, the sweep, the argmax; for accounting). */
int mld_decode_launches(void);

/* Static description of a status code. */
const char* mld_status_string(mld_status s);

#ifdef __cplusplus
}
#endif

#endif /* MLD_H */
