/*
 * shape.h -- C ABI of libshape: importance-sampling estimation of Gaussian
 * molecular shape overlap on one B300 GPU (sm_103a).
 *
 * Method: Tuzharov, Bochenkova, Maximov, "Importance-Sampling Estimation of
 * Gaussian Molecular Shape Overlap: Exact Union Volumes and
 * Confidence-Bounded Virtual Screening" (arXiv 2607.20766).
 *
 * Conventions for every entry point
 *   - Return value: SHP_OK (0) or a negative status; shp_last_error() gives
 *     a message for the calling thread. No exception crosses the ABI.
 *   - Pointers named *_host are host memory. Every other array argument is
 *     DEVICE memory owned by the caller (e.g. a torch CUDA tensor), on the
 *     current device, and must stay valid until the work queued on `stream`
 *     has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Arguments are checked synchronously; GPU work is queued
 *     asynchronously on `stream` and results are ready when the stream is.
 *   - A shp_set is immutable after shape_set_load; concurrent calls on
 *     different streams may share it. shape_set_free must not race with
 *     work that still uses the set.
 *   - Molecules hold 1..SHP_MAX_ATOMS atoms (else SHP_ERANGE).
 *
 * Model (Eq. occ, Eq. union, Sec. first-order overlap): atom i has centre
 * c_i, radius R_i, height p_i (default 2 sqrt 2) and
 * alpha_i = c_alpha / R_i^2 (default c_alpha = 2.41798793); its Gaussian is
 * g_i(r) = p_i exp(-alpha_i |r - c_i|^2). m(r) = sum_i g_i(r) is the
 * first-order density and u(r) = 1 - prod_i (1 - g_i(r)) the union
 * occupancy. Z = sum_i p_i (pi / alpha_i)^{3/2} = integral of m.
 *
 * Random streams: counter-based Philox4x32-10, key = seed, counter =
 * (block, stream lo, stream hi, tag); the sample layout is fixed so that any
 * independent implementation of the same specification reproduces every
 * sample (see the library's design notes).
 */
#ifndef SHAPE_H
#define SHAPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHP_OK 0
#define SHP_EINVAL (-1)   /* bad argument (NULL, negative size, NaN, ...)   */
#define SHP_ENOMEM (-2)   /* device or host allocation failed               */
#define SHP_ECUDA (-3)    /* a CUDA runtime call failed                      */
#define SHP_ERANGE (-4)   /* atom count outside 1..SHP_MAX_ATOMS, index out of range */
#define SHP_ETIMEOUT (-5) /* reserved for a bounded device-side wait that gives
                             up; no entry point returns it: no kernel of the
                             library waits on another block or on the host   */

#define SHP_MAX_ATOMS 64

/* Monte-Carlo flags */
#define SHP_SYMMETRIC 1u  /* estimate from both proposals and average (Sec. IS estimator) */
#define SHP_ANTITHETIC 2u /* pair each draw with its reflection about the component centre */
#define SHP_ID_STREAMS 4u /* per-molecule calls with an idx list: molecule idx[k] draws from stream
                             stream_base + idx[k] (its id) instead of stream_base + k, so the
                             listed molecules get exactly the values of a call over the whole set */

/* Stream tags (counter word 3) */
#define SHP_TAG_AB 0u   /* samples drawn from A's mixture, B evaluated */
#define SHP_TAG_BA 1u   /* samples drawn from B's mixture, A evaluated */
#define SHP_TAG_SELF 2u /* a molecule's own volume / self-overlap      */

typedef struct shp_set_s* shp_set;

/* Message of the last failing call on this host thread ("" if none). */
const char* shp_last_error(void);

/* ABI version (incremented on any signature change). */
int shp_version(void);

/*
 * Test hook: the next `count` device allocations made by library calls fail
 * as out of memory (the call returns SHP_ENOMEM with a message, having
 * released what it had allocated) without calling CUDA; 0 clears the hook.
 * Lets callers exercise their error paths on the host. SHP_EINVAL for a
 * negative count.
 */
int shp_fail_next_allocations(int32_t count);

/*
 * Load n_mol molecules into device memory (Eq. occ, Eq. expectation).
 *   xyz_host      [n_atoms][3] float, Angstrom (n_atoms = offsets_host[n_mol])
 *   radius_host   [n_atoms] float > 0, Angstrom
 *   height_host   [n_atoms] float > 0, or NULL for 2 sqrt 2
 *   c_alpha       alpha_i = c_alpha / R_i^2; <= 0 selects 2.41798793
 *   offsets_host  [n_mol + 1] int32, offsets_host[0] = 0, non-decreasing,
 *                 every count in 1..SHP_MAX_ATOMS
 *   n_mol         >= 0
 * Builds per molecule the mixture mass Z, the integer alias table of the
 * component probabilities v_i / Z, and a largest-first order used to
 * balance screens. The host threads (OpenMP) validate the inputs and pack
 * coordinates, radii (and heights) into a staging buffer; one copy uploads
 * them (20 B per atom, 24 with heights) on a library-owned upload stream,
 * where a kernel then computes alpha, the sampling width, log2 p, the
 * volumes v_i = p_i (pi / alpha_i)^{3/2}, Z and the alias tables in FP64
 * with IEEE-rounded operations (log2 p of given heights by CUDA's FP64
 * log2). `stream` is made to wait for that work (work enqueued on `stream`
 * after the call sees the set, while kernels already queued on it overlap
 * the copy; other streams must order themselves after `stream`).
 * Not capturable into a CUDA graph. The host arrays may be reused as soon as the
 * call returns (they are copied into one of two library-owned pinned
 * staging buffers, and a call waits only for the upload made from the same
 * buffer two calls earlier). On success *out owns all device memory of the
 * set (free with shape_set_free or shape_set_free_async). Errors: SHP_EINVAL (NULL, non-finite or non-positive
 * values), SHP_ERANGE (atom counts), SHP_ENOMEM, SHP_ECUDA.
 */
int shape_set_load(const float* xyz_host, const float* radius_host, const float* height_host,
                   double c_alpha, const int32_t* offsets_host, int32_t n_mol, void* stream,
                   shp_set* out);

/* Free a set (NULL is a no-op). Synchronises the device first. */
int shape_set_free(shp_set s);

/*
 * Free a set in stream order (NULL is a no-op): its device memory returns to
 * the pool once the work enqueued on `stream` before this call has run. The
 * caller guarantees that no work on another stream still uses the set. Does
 * not synchronise.
 */
int shape_set_free_async(shp_set s, void* stream);

/* Sizes of a set; any output may be NULL. */
int shape_set_info(shp_set s, int32_t* n_mol, int64_t* n_atoms, int32_t* max_atoms);

/*
 * Host copies of the per-molecule mixture masses Z ([n_mol] double) and of
 * the alias tables ([n_atoms] uint32 thresholds, [n_atoms] uint8 aliases,
 * indices local to each molecule). Any output may be NULL. The tables are
 * read back from the device (synchronises it).
 */
int shape_set_tables(shp_set s, double* Z_host, uint32_t* thr_host, uint8_t* alias_host);

/* Monte-Carlo settings shared by the estimators. */
typedef struct {
  uint64_t seed;        /* Philox key                                        */
  uint64_t stream_base; /* item k uses Philox stream stream_base + k          */
  uint32_t n_samples;   /* per direction, >= 2 (even with SHP_ANTITHETIC)     */
  uint32_t flags;       /* SHP_SYMMETRIC | SHP_ANTITHETIC                      */
} shp_mc;

/*
 * Pair overlaps by importance sampling (Eq. expectation, Eq. var,
 * Eq. union-is). For pair k, molecule A[ia[k]] and B[ib[k]] moved by
 * poseB[k] (unit-normalised quaternion w,x,y,z then translation; NULL =
 * identity): draws n_samples points from A's mixture (tag SHP_TAG_AB) and,
 * with SHP_SYMMETRIC, n_samples from the posed B's mixture (tag
 * SHP_TAG_BA), and writes
 *   est[k][0], se[k][0]   first-order overlap  Z_A mean(m_B)
 *   est[k][1], se[k][1]   union overlap        Z_A mean(u_A u_B / m_A)
 * (symmetrised: mean of the two directions, SE 0.5 sqrt(se_AB^2 + se_BA^2)).
 * SE = Z sqrt(s^2 / n) with the n-1 sample variance; with SHP_ANTITHETIC the
 * unit is the mean of a reflected pair.
 *   ia, ib   [n_pairs] int32 device;  poseB [n_pairs][7] float device or NULL
 *   est, se  [n_pairs][2] double device
 * Errors: SHP_EINVAL, SHP_ECUDA; out-of-range indices are not checked on
 * the host (the kernel skips them and leaves their outputs as NaN).
 */
int overlap_estimate(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
                     const float* poseB, const shp_mc* mc, double* est, double* se, void* stream);

/*
 * Union volume and union self-overlap of molecules S[idx[k]] (Eq. union-is
 * with f = u/m, and with B = A): samples from the molecule's own mixture
 * (tag SHP_TAG_SELF, stream mc->stream_base + k) and writes
 *   vol[k], vol_se[k]         V = Z mean(u/m)
 *   self_ov[k], self_se[k]    O_AA = Z mean(u^2/m)   (both may be NULL)
 *   idx   [n] int32 device or NULL (= 0..n-1); outputs [n] double device.
 * mc->flags: SHP_ANTITHETIC, SHP_ID_STREAMS (stream mc->stream_base + idx[k]).
 */
int union_volume_estimate(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, double* vol,
                          double* vol_se, double* self_ov, double* self_se, void* stream);

/*
 * Closed-form first-order overlap (Eq. fo with heights):
 *   out[k] = sum_{i in A, j in B} p_i p_j (pi/(a_i+a_j))^{3/2}
 *            exp(-a_i a_j / (a_i + a_j) |c_i - c'_j|^2)
 * with c'_j the centres of B[ib[k]] moved by poseB[k] (NULL = identity).
 *   ia, ib [n_pairs] int32 device; poseB [n_pairs][7] float or NULL;
 *   out [n_pairs] double device.
 */
int fo_overlap(shp_set A, const int32_t* ia, shp_set B, const int32_t* ib, int64_t n_pairs,
               const float* poseB, double* out, void* stream);

/*
 * First-order Tanimoto of every pair (Q[q], D[d]) in closed form (Eq. fo
 * with heights; Sec. union for the Tanimoto):
 *   T_fo[q * n_db + d] = O / (S_q + S_d - O),
 *   O = sum_{i in Q[q], j in D[d]} p_i p_j (pi/(a_i+a_j))^{3/2}
 *       exp(-a_i a_j / (a_i+a_j) |c_i - c_j|^2)
 * with S the same closed form of a molecule with itself (fo_overlap of the
 * molecule with itself). The cheap first stage of the paper's hybrid
 * pipeline, used to drop clear misses before the union screen. Terms and the
 * per-pair sum in FP32: each term as w_i w_j r^3 2^(-r^2 |c_i - c_j|^2) with
 * r = (1/(a_i log2 e) + 1/(a_j log2 e))^(-1/2) and per-atom weights w (SFU
 * rsqrt and exp2 per atom pair, SFU log2 and reciprocal per atom).
 *   fo_self_q [n_q], fo_self_db [n_db] double device; T_fo [n_q * n_db]
 *   float device. At most 65535 queries per call (SHP_ERANGE).
 */
int fo_tanimoto_screen(shp_set Q, shp_set D, const double* fo_self_q, const double* fo_self_db, float* T_fo,
                       void* stream);

/*
 * Selection step of the first-order prefilter: for every query q the k
 * database molecules with the largest scores T[q * n_db + d] (e.g.
 * fo_tanimoto_screen's output), exactly: every score above the k-th largest
 * is kept, and of the scores equal to it the lowest database ids until k.
 * Writes the pair list of tanimoto_screen, per query in ascending database
 * id: pairs_q[q * k + j] = q, pairs_db[q * k + j] = d. Deterministic (a
 * radix select on the FP32 scores' order-preserving 32-bit keys, three
 * passes of 12, 12 and 8 bits). Scores must not be NaN.
 *   T [n_q * n_db] float device; pairs_q, pairs_db [n_q * k] int32 device;
 *   1 <= k <= n_db (else SHP_ERANGE), at most 65535 queries.
 * Scratch (per-query histograms and per-chunk counts) is stream-ordered
 * library memory.
 */
int fo_prefilter_select(shp_set Q, shp_set D, const float* T, int64_t k, int32_t* pairs_q, int32_t* pairs_db,
                        void* stream);

/*
 * The database molecules a pair list keeps (e.g. fo_prefilter_select's
 * pairs_db), as an idx list for the per-molecule calls: ids[d] = d for every
 * d listed at least once, -1 for the rest. Passed as idx (with
 * SHP_ID_STREAMS) to union_self_estimate or cv_fit_weights, it computes the
 * kept molecules only, each with exactly the values of a call over the whole
 * set, at position d of the outputs (the -1 entries are skipped: NaN
 * estimates, no weights written).
 *   pairs_db [n_pairs] int32 device (ids outside the set are ignored);
 *   ids [n_db] int32 device, written.
 */
int prefilter_db_ids(shp_set D, const int32_t* pairs_db, int64_t n_pairs, int32_t* ids, void* stream);

/* Screening settings (Sec. confidence-bounded screening). */
typedef struct {
  uint64_t seed;        /* Philox key                                              */
  uint64_t stream_base; /* pair (q, d) uses stream stream_base + q * stride + d     */
  uint32_t n_fixed;     /* > 0: fixed budget, samples per direction (>= 2);
                           0: adaptive (fields below)                              */
  uint32_t flags;       /* SHP_ANTITHETIC (fixed budget only; both directions are
                           always used)                                            */
  float tau;            /* adaptive: stop a pair once SE(T) <= tau                 */
  uint32_t round;       /* adaptive: samples per direction per round, a multiple
                           of 256                                                  */
  uint32_t min_n;       /* adaptive: first check after min_n samples per direction
                           (a multiple of round, >= round)                         */
  uint32_t cap;         /* adaptive: at most cap samples per direction (a multiple
                           of round, >= min_n)                                     */
  uint32_t watch;       /* adaptive: which Tanimoto the rule watches, 1 = union,
                           0 = first order                                         */
  int32_t variant;      /* launch variant, -1 = the tuned (or built-in) default,
                           else 0 .. shp_screen_variants()-1                      */
  const float* omega_q; /* control variate of the union slot: per-atom weights of
                           Q and of D (device, set atom order), both or neither;
                           NULL = plain estimator                                  */
  const float* omega_db;
  const double* self_se_q;  /* standard errors of self_q / self_db ([n][2] device,
                               same layout), both or neither; NULL = the
                               self-overlaps are exact                             */
  const double* self_se_db;
  uint64_t stream_stride;   /* the stride above; 0 = n_db. A database shard
                               [start, end) of a global database of n_global
                               molecules uses stream_base = start and stride =
                               n_global, and reproduces the global screen's
                               numbers for its pairs                        */
  const int32_t* pairs_q;   /* optional explicit pair list (device int32
                               [n_pairs], both or neither): only the pairs
                               (pairs_q[k], pairs_db[k]) are screened and the
                               outputs are indexed by k; streams stay keyed by
                               (q, d), so each listed pair gets the numbers
                               the full screen would give it. NULL (with
                               n_pairs 0) = every pair of Q x D; an empty list
                               is not expressible, skip the call instead     */
  const int32_t* pairs_db;
  int64_t n_pairs;
} shp_screen;

/*
 * Tanimoto screen of every query Q[q] against every database molecule D[d]
 * (Sec. confidence-bounded screening). Both proposals give the symmetrised
 * first-order and union overlaps O; with the self-overlaps S_Q, S_D supplied
 * by the caller (slot 0 first order, slot 1 union, e.g. fo_overlap of a
 * molecule with itself and union_volume_estimate's self_ov), writes for pair
 * p = q * n_db + d and slot s:
 *   T[p][s]   = O / (S_Q + S_D - O)
 *   seT[p][s] = (S_Q + S_D) / (S_Q + S_D - O)^2 * SE(O)   (delta method)
 * and, when the self-overlaps are estimates with standard errors
 * cfg->self_se_q, cfg->self_se_db (e.g. union_self_estimate's self_se), the
 * full delta-method SE of T(O, S_Q, S_D), whose terms are independent:
 *   seT^2 = ((S_Q + S_D) / den^2 SE(O))^2 + (O / den^2)^2 (se_Q^2 + se_D^2),
 *   den = S_Q + S_D - O
 *   O_out[p][s], seO_out[p][s] (double, may be NULL)
 *   n_used[p] samples drawn per direction (may be NULL)
 * Control variate (omega_q, omega_db given): the union overlap is estimated
 * as C + Z E_q[(u_A u_B - u~_A u~_B) / m_A] per direction, u~ = sum_i w_i g_i,
 * with C = sum_ij w_i w_j integral g_i g_j in closed form (Eq. fo with
 * weights): unbiased for any weights; the first-order slot is unchanged.
 * Fixed budget: n_fixed samples per direction. Adaptive (n_fixed == 0):
 * rounds of `round` samples per direction are drawn until, after at least
 * min_n, the watched SE(T) (computed in FP32 from the running sums, and
 * the full SE when self-overlap SEs are given) is <= tau, or cap is reached;
 * the samples are the first n_used of the same streams a fixed budget would
 * draw.
 *   self_q [n_q][2], self_db [n_db][2] double device
 *   T, seT [n_q * n_db][2] (or [n_pairs][2] with a pair list) float device
 * Work is balanced by a persistent kernel that takes pairs largest-first
 * from a device queue (library-allocated, stream-ordered scratch); a pair
 * list is taken in its own order (list large molecules first). Indices of a
 * pair list outside the sets are skipped (their outputs are not written).
 */
int tanimoto_screen(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q,
                    const double* self_db, float* T, float* seT, double* O_out, double* seO_out,
                    uint32_t* n_used, void* stream);

/*
 * Roofline calibration (a measurement aid; the paper has none): runs the
 * per-sample work of screen launch variant `variant` (-1 = the tuned
 * default) on the pair (Q[iq], D[id]) -- every atom of both molecules
 * evaluated at each sample and the per-lane accumulation, both directions --
 * on as many warps as the variant keeps resident, `batches` batches of 64 SP
 * samples per direction per warp, with no pair queue and no per-pair
 * epilogue. draw = 1: the samples are drawn as in the screen (Philox words,
 * alias pick, Box-Muller normals); draw = 0: they are placed at the staged
 * component centres moved by a per-batch offset, i.e. the same position
 * arithmetic without the random draw. *evals_host receives the sample x atom
 * evaluations one call performs; time it with events on `stream`.
 *   sink [1] double device: a checksum is added to it (keeps the work live).
 * Errors: SHP_EINVAL, SHP_ERANGE (indices, variant), SHP_ECUDA.
 */
int shp_eval_probe(shp_set Q, int32_t iq, shp_set D, int32_t id, int32_t variant, int32_t draw,
                   uint32_t batches, double* sink, int64_t* evals_host, void* stream);

/* Number of compiled launch variants of the screen kernel. */
int shp_screen_variants(void);

/*
 * Shape of launch variant v: info[0] sample pairs per lane per batch (the
 * adaptive screen runs only the variants with 4), info[1] exponent/loop form,
 * info[2] warps per CTA, info[3] CTAs per SM the register budget is set for.
 * Returns SHP_ERANGE for v outside 0 .. shp_screen_variants()-1, SHP_EINVAL
 * for a NULL info.
 */
int shp_screen_variant_info(int32_t v, int32_t info[4]);

/*
 * Autotuner: times every launch variant valid for cfg (fixed or adaptive) on
 * n_sample pairs spread evenly over the screen (outputs go to the caller's
 * T/seT/n_used buffers), makes the fastest the default of this device for
 * that mode, and returns its id in *best. timings_ms [shp_screen_variants()]
 * receives each variant's time (or -1 if not valid); may be NULL.
 * Synchronises `stream`.
 */
int tanimoto_screen_tune(shp_set Q, shp_set D, const shp_screen* cfg, const double* self_q,
                         const double* self_db, float* T, float* seT, uint32_t* n_used,
                         int64_t n_sample, float* timings_ms, int32_t* best, void* stream);

/* ---------------------------------------------------------------------- */
/* Rigid alignment (Sec. differentiable alignment, Eq. pose, Eq. grad)     */
/* ---------------------------------------------------------------------- */

#define SHP_TAG_CRN 3u   /* common-random-number points of a query      */
#define SHP_TAG_START 4u /* random starting rotations of align_rigid     */
#define SHP_OBJ_FO 0u    /* CRN objective (Z_Q/n) sum_k m_B(r_k)        */
#define SHP_OBJ_UNION 1u /* CRN objective (Z_Q/n) sum_k w_k u_B(r_k)    */
#define SHP_OBJ_FO_CLOSED 2u /* closed-form first-order overlap (Eq. fo): the
                                exact, deterministic objective of the paper's
                                hybrid pipeline (align on first order, score on
                                the union); the CRN points are not used      */

/*
 * Common random numbers: mc->n_samples points drawn from Q[iq]'s mixture
 * (tag SHP_TAG_CRN, stream mc->stream_base, the usual sample layout) with
 * their union weights: points [n][4] float device = (x, y, z, u_Q/m_Q).
 * mc->flags: 0 or SHP_ANTITHETIC (each odd point the reflection of the even
 * one about its component centre, Sec. IS estimator's antithetic pairs).
 */
int align_crn_points(shp_set Q, int32_t iq, const shp_mc* mc, float* points, void* stream);

/*
 * Fused forward/adjoint of the CRN overlap (Eq. grad) for items k: molecule
 * B[ib[k]] moved by pose[k] = (raw quaternion w, x, y, z -- normalised
 * inside --, translation), the n_points CRN points of Q[iq]:
 *   value[k] = (Z_Q / n) sum_j f(r_j),  f = m_B (SHP_OBJ_FO) or w_j u_B
 *              (SHP_OBJ_UNION)
 *   grad[k][7] = d value[k] / d pose[k]  (through the normalisation)
 * The union derivative is w q g_j / f_j with f_j = 1 - g_j rounded once and
 * q the product of the same rounded f_l, so the quotient is the product over
 * l != j to rounding (an f_j of exactly 0 is replaced by 2^-100).
 *   points [n_points][4] float, ib [n_items] int32, pose [n_items][7] float,
 *   value [n_items] double, grad [n_items][7] float; all device.
 */
int overlap_pose_grad(shp_set Q, int32_t iq, const float* points, uint32_t n_points, shp_set B,
                      const int32_t* ib, int64_t n_items, const float* pose, uint32_t objective,
                      double* value, float* grad, void* stream);

/* Multi-start alignment settings. */
typedef struct {
  uint64_t seed;      /* Philox key for CRN points, random starts and scoring      */
  uint64_t stream;    /* Philox stream of the CRN points and scoring base           */
  uint32_t starts;    /* starts per pair, 1..64: 4 principal-axis sign patterns,
                         then uniform random rotations                              */
  uint32_t steps;     /* Adam steps                                                 */
  uint32_t n_crn;     /* CRN points per step                                        */
  uint32_t objective; /* SHP_OBJ_FO or SHP_OBJ_UNION                                */
  float lr, lr_t;     /* Adam step sizes of the quaternion and of the translation   */
  float beta1, beta2, eps;
  uint32_t n_score;   /* samples per direction for the final union Tanimoto          */
  uint32_t crn_flags; /* 0 or SHP_ANTITHETIC: the CRN points in antithetic pairs
                         (align_crn_points), the same number of points            */
} shp_align;

/*
 * Multi-start rigid alignment of database molecules B[ib[k]] onto the query
 * Q[iq] (Sec. differentiable alignment): per pair, `starts` poses (B's
 * principal frame mapped onto Q's with the four proper sign patterns, then
 * random rotations between the frames, centroids matched), `steps` Adam
 * ascent steps on the CRN objective (step sizes decayed by
 * (1 + cos(pi step / steps)) / 2), then each final pose is scored by the
 * symmetrised union Tanimoto (overlap_estimate with n_score samples and the
 * union self-overlaps self_q[iq][1], self_db[ib[k]][1]; every start of pair
 * k on the same random numbers, stream cfg->stream + k, seed cfg->seed ^
 * 0x5DEECE66D, so that starts are compared on common random numbers) and
 * the best start is kept.
 *   self_q [n_q][2], self_db [n_db][2] double device (slot 1 = union)
 *   pose_out [n_pairs][7], T_out [n_pairs], T_starts [n_pairs][starts]
 *   (may be NULL), pose_starts [n_pairs][starts][7] (the final raw pose of
 *   every start, may be NULL) float device.
 * Scratch (CRN points, per-start poses, scores) is stream-ordered library
 * memory.
 */
int align_rigid(shp_set Q, int32_t iq, shp_set B, const int32_t* ib, int64_t n_pairs,
                const shp_align* cfg, const double* self_q, const double* self_db, float* pose_out,
                float* T_out, float* T_starts, float* pose_starts, void* stream);

/* ---------------------------------------------------------------------- */
/* Learned control variate for union volumes                               */
/* ---------------------------------------------------------------------- */
/*
 * Not in the paper: a per-atom network predicts crowding weights om_i; the
 * weighted Gaussians u~ = sum_i om_i g_i have the closed-form volume
 * sum_i om_i v_i (v_i = p_i (pi/alpha_i)^{3/2}), and the sampler estimates
 * only the residual, V = sum_i om_i v_i + Z E_q[(u - u~)/m] -- unbiased for
 * any om (Eq. expectation with f = (u - u~)/m).
 */

#define SHP_TAG_ATTR 5u /* samples of the union attributions */
#define SHP_TAG_FIT 6u  /* samples of the least-squares control-variate fit */

/*
 * Union attributions om*_i = E_{r ~ N(c_i, I/(2 alpha_i))}[u(r)/m(r)] for
 * every atom of S (training targets of the network; sum_i v_i om*_i = V):
 * M samples per atom (a multiple of 256); atom i of molecule k uses sample
 * pairs i M/2 .. (i+1) M/2 - 1 of stream stream_base + k, tag SHP_TAG_ATTR,
 * normals only. omega [n_atoms] float device.
 */
int union_attributions(shp_set S, uint64_t seed, uint64_t stream_base, uint32_t M, float* omega,
                       void* stream);

/*
 * Least-squares control-variate weights (not in the paper; for the screen's
 * union slot): for molecule k of the list the weights w minimising the
 * integral of (u - sum_i w_i g_i)^2, the projection of the union occupancy
 * onto the molecule's own Gaussians:
 *   (G + lambda I) w = b,   G_ij = integral g_i g_j (closed form, Eq. fo terms),
 *   b_i = integral u g_i = Z E_q[(u / m) g_i],   lambda = ridge * trace(G) / N,
 * b from mc->n_samples (a positive multiple of 256) samples of the molecule's
 * own mixture (stream mc->stream_base + k, tag SHP_TAG_FIT, the usual sample
 * layout; mc->flags: 0 or SHP_ID_STREAMS, then stream mc->stream_base +
 * idx[k]), solved by conjugate gradients to a relative
 * residual of 1e-6 (at most 4 N iterations).
 *   idx [n] device int32 molecule ids, or NULL for molecules 0 .. n-1
 *   omega [n_atoms] float device: written for the atoms of the listed
 *   molecules (set atom order); other entries are left as they are. An id
 *   outside 0 .. n_mol-1 (not checked on the host: idx is device memory)
 *   is skipped and writes nothing.
 * The conjugate-gradient iteration stops early, keeping its last finite
 * iterate, if a step becomes non-finite or the curvature p.Gp is not
 * positive (possible for ridge = 0 and nearly coincident atoms).
 * Errors: SHP_EINVAL (NULL, bad n_samples, flags or ridge), SHP_ERANGE.
 */
int cv_fit_weights(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, float ridge, float* omega,
                   void* stream);

/*
 * Union volume of molecules S[idx[k]] with the control variate omega (per
 * set atom, float device; NULL = plain estimator), same samples as
 * union_volume_estimate (tag SHP_TAG_SELF, stream mc->stream_base + k, or
 * + idx[k] with mc->flags = SHP_ID_STREAMS; no other flags).
 * target_rel_se <= 0: mc->n_samples samples. target_rel_se > 0: rounds of
 * `round` samples (a multiple of 256 dividing mc->n_samples, which is then
 * the cap) until SE / V <= target_rel_se (checked in FP32).
 *   vol, vol_se [n] double, n_used [n] uint32 (may be NULL); device.
 */
int union_volume_cv(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, const float* omega,
                    float target_rel_se, uint32_t round, double* vol, double* vol_se, uint32_t* n_used,
                    void* stream);

/*
 * Union volumes and union self-overlaps of molecules S[idx[k]] to a stated
 * precision (Eq. expectation with f = u/m and Eq. union-is with B = A; the
 * self-overlaps are the O_AA of the Tanimoto, Sec. union). Same samples as
 * union_volume_estimate (tag SHP_TAG_SELF, stream mc->stream_base + k, or
 * + idx[k] with mc->flags = SHP_ID_STREAMS; no other flags). With omega (per set atom, float device; NULL = plain) both carry
 * the weighted-Gaussian control variate u~ = sum_i omega_i g_i:
 *   V    = sum_i omega_i v_i                  + Z E_q[(u - u~) / m]
 *   O_AA = sum_ij omega_i omega_j int g_i g_j + Z E_q[(u^2 - u~^2) / m]
 * (not in the paper; unbiased for any omega). target_rel_se <= 0:
 * mc->n_samples samples. target_rel_se > 0: rounds of `round` samples (a
 * multiple of 256 dividing mc->n_samples, which is then the cap) until the
 * watched estimate (watch 0: volume, 1: self-overlap) has SE / estimate <=
 * target_rel_se, checked in FP32 after each round.
 *   idx [n] int32 device or NULL (= 0..n-1); vol, vol_se, self_ov, self_se
 *   [n] double and n_used [n] uint32 device, each may be NULL (not both vol
 *   and self_ov).
 * Errors: SHP_EINVAL, SHP_ERANGE, SHP_ENOMEM, SHP_ECUDA.
 */
int union_self_estimate(shp_set S, const int32_t* idx, int64_t n, const shp_mc* mc, const float* omega,
                        float target_rel_se, uint32_t round, uint32_t watch, double* vol, double* vol_se,
                        double* self_ov, double* self_se, uint32_t* n_used, void* stream);

#define SHP_MLP_IN 33
#define SHP_MLP_HIDDEN 64
#define SHP_MLP_PARAMS 6401 /* W1 64x33, b1 64, W2 64x64, b2 64, w3 64, b3 1 */

/*
 * Per-atom features of every atom of S: the 16 nearest other atoms of the
 * molecule by distance (ties by index) as (d / 4 A, R / 1.7 A) pairs, then
 * the atom's own R / 1.7 A; missing neighbours are (2.5, 0).
 * feat [n_atoms][33] float device.
 */
int cv_features(shp_set S, float* feat, void* stream);

/*
 * The network: z1 = W1 x + b1, h1 = GELU(z1), z2 = W2 h1 + b2,
 * h2 = GELU(z2), y = w3 . h2 + b3 (GELU in the erf form). params
 * [SHP_MLP_PARAMS] float device is the FP32 master copy in the order above
 * (matrices row-major); the kernels compute with the parameters rounded to
 * BF16 and accumulate in FP32.
 * mlp_forward: y[k] for the rows rows[k] of x (rows NULL = 0..n-1).
 *   x [*][33] float, y [n] float; device.
 */
int mlp_forward(const float* params, const float* x, const int32_t* rows, int64_t n, float* y,
                void* stream);

/*
 * Loss L = mean_k (y_k - target[rows[k]])^2 over the selected rows and its
 * gradient with respect to the (BF16-rounded) parameters, reduced
 * deterministically: grad [SHP_MLP_PARAMS] float, loss [1] double; device.
 * Scratch (per-block partial gradients) is stream-ordered library memory.
 */
int mlp_loss_grad(const float* params, const float* x, const float* target, const int32_t* rows,
                  int64_t n, float* grad, double* loss, void* stream);

/*
 * mlp_loss_grad without any device allocation (the paper has no
 * counterpart). For callers that cannot allocate device memory while they
 * run -- a host framework that owns the device allocator and forbids
 * allocation inside its training step, or a latency-bound loop that cannot
 * take an allocation. Same arguments, outputs and results as mlp_loss_grad;
 * the per-block partial gradients go to a fixed array inside the library
 * (128 x 6402 floats, 3.3 MB held on every device that loads the library
 * until the process exits), so a call takes at most 8192 rows: larger n
 * returns SHP_ERANGE. The first call on each device looks up the array's
 * device address (make that first call before any stream capture). A call
 * overwrites the part of the array it uses, so nothing carries over between
 * calls; calls that overlap on the GPU (e.g. on two streams) race on it.
 * The looked-up address is kept for the life of the process: after a
 * cudaDeviceReset of that device the library must not be called on it again
 * (the cached address would then be stale).
 */
int mlp_loss_grad_noalloc(const float* params, const float* x, const float* target,
                          const int32_t* rows, int64_t n, float* grad, double* loss, void* stream);

/*
 * One Adam descent step on the FP32 master parameters (step >= 1, bias
 * corrected): m, v [n_params] float device moments, updated in place.
 */
int mlp_adam(float* params, float* m, float* v, const float* grad, int64_t n_params, int64_t step,
             float lr, float beta1, float beta2, float eps, void* stream);

/*
 * One epoch of minibatch training in one call: for each minibatch of
 * `batch` rows of perm (the last one may be shorter), mlp_loss_grad on those
 * rows, then mlp_adam with step step0 + 1, step0 + 2, ... The launches are
 * those of the step-by-step calls, in the same order, so the parameters and
 * moments end exactly as theirs; the host loop runs inside the library.
 *   params, m, v [SHP_MLP_PARAMS] float device, updated in place;
 *   x [*][SHP_MLP_IN], target [*] float device; perm [n] int32 device rows;
 *   losses [ceil(n / batch)] double device: each minibatch's mean squared error.
 * Scratch (partial gradients, the gradient) is stream-ordered library memory.
 */
int mlp_train_epoch(float* params, float* m, float* v, const float* x, const float* target, const int32_t* perm,
                    int64_t n, int64_t batch, int64_t step0, float lr, float beta1, float beta2, float eps,
                    double* losses, void* stream);

/*
 * Host copy of each molecule's principal frame ([n_mol][12] float: the
 * Gaussian-volume-weighted centroid, then the 3x3 axis matrix row-major with
 * the axes as columns, sorted by decreasing second moment, the first two
 * oriented to a non-negative third moment, det +1), read back from the
 * device (synchronises it).
 */
int shape_set_frames(shp_set s, float* frames_host);

#ifdef __cplusplus
}
#endif

#endif /* SHAPE_H */
