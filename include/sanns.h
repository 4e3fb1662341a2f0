/*
 * sanns.h -- C ABI of libsanns.so, the B300 (sm_103a) implementation of the
 * server-side hot path of SANNS (Chen et al., "SANNS: Scaling Up Secure
 * Approximate k-Nearest Neighbors Search", arxiv 1904.02033): homomorphic
 * evaluation of query-to-point squared distances under RNS BFV.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Buffers named *_dev are device memory of the current CUDA device (for
 *   instance a torch tensor's data_ptr()); *_host are host memory; "any" means
 *   either (copied with cudaMemcpyDefault).  The caller owns every buffer it
 *   passes; opaque handles (sanns_ctx, sanns_sk, sanns_db, sanns_clusters,
 *   sanns_gather_batch) are owned by the library and released with the
 *   matching sanns_*_free.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls enqueue work on it and return without synchronising unless stated;
 *   buffers must stay alive until the stream has passed the call.
 * - Residues are uint64 in [0, q_j).  Ciphertext polynomials are laid out
 *   [..][2][L][N]: component c0/c1, prime j, coefficient/slot.  "NTT form"
 *   means slot s holds the evaluation at psi_j^(2 brv(s) + 1).
 * - Every call returns SANNS_OK (0) or a negative code; the message of the
 *   last failure on the calling thread is sanns_last_error().  Arguments are
 *   validated on the host before anything is launched; an invalid argument
 *   launches nothing.
 * - Host threads: the computing calls keep no state in a handle (their
 *   scratch is allocated stream-ordered per call), so several threads may
 *   call them on one context and database at once, each with its own stream
 *   and output buffers.  Calls that change a handle's settings or contents
 *   (sanns_set_*, sanns_autotune_*, sanns_batched_tune,
 *   sanns_db_prepare_batched, sanns_db_set_position_base, the *_free calls)
 *   must not overlap any other call on that handle.  The device error word
 *   read by sanns_device_status is shared by all calls on a context.  The
 *   one exception to the no-shared-state rule is
 *   sanns_decrypt_shares_noalloc: its scratch is one process-wide array per
 *   device, shared by every context on that device, so its calls on one
 *   device must be ordered (one stream, or events between streams).
 *
 * Readings of the paper that fix the exact bits (the paper leaves them to
 * SEAL): primes = the L largest primes below 2^prime_bits that are 1 mod 2N;
 * psi_j = the smallest primitive 2N-th root of unity; Delta = floor(Q/t);
 * randomness = ChaCha20 (RFC 8439) streams keyed by a 64-bit seed.
 */
#ifndef SANNS_H_
#define SANNS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SANNS_OK 0
#define SANNS_EINVAL (-1)   /* bad shape, parameter or pointer */
#define SANNS_ENOMEM (-2)   /* device allocation failed */
#define SANNS_ECUDA (-3)    /* a CUDA call failed; see sanns_last_error() */
#define SANNS_ETIMEOUT (-4) /* a bounded device-side wait gave up */

typedef struct sanns_ctx sanns_ctx;
typedef struct sanns_sk sanns_sk;
typedef struct sanns_db sanns_db;
typedef struct sanns_clusters sanns_clusters;
typedef struct sanns_gather_batch sanns_gather_batch;

/*
 * BFV parameters (Sec. 7.1 "Parameter choices": N = 2^13, 180-bit q as three
 * machine words, t = 2^b_d; Fig. "hyperparameters": b_d = 2 b_c + ceil(log2 d)).
 *   N           ring degree, a power of two in [64, 16384]
 *   L           number of RNS primes, 1..4
 *   prime_bits  bit size of each prime, 20..60
 *   t_rule      0: t = smallest prime > 2^24 with t = 1 mod 2N;
 *               1: t = 2^(2 b_c + ceil(log2 d)) as in the paper
 *   d           vector dimension, 1..224
 *   b_c         coordinate bits for t_rule 1 (coordinates are uint8 here)
 */
typedef struct {
  uint32_t N, L, prime_bits, t_rule, d, b_c;
} sanns_params;

const char *sanns_last_error(void);

/* Derive primes, psi, t, Delta and the twiddle tables; upload them to the
 * current device.  Synchronous.  *out is NULL on failure. */
int sanns_ctx_create(const sanns_params *params, sanns_ctx **out);
void sanns_ctx_free(sanns_ctx *ctx);
/* Read back derived values (host arrays of L entries; any pointer may be
 * NULL). */
int sanns_ctx_query(const sanns_ctx *ctx, uint64_t *q_host, uint64_t *psi_host, uint64_t *t_host,
                    uint64_t *delta_host);

/*
 * In-place negacyclic NTT (inverse != 0: inverse NTT) of `count` groups of L
 * polynomials, data_dev laid out [count][L][N]; polynomial (g, j) uses prime
 * j.  Inputs must be canonical; outputs are canonical.  The transform the
 * ct x pt product is taken through (Sec. 5.3's products g_i f_i live in
 * R_q = Z_q[x]/(x^N + 1)).
 */
int sanns_ntt(sanns_ctx *ctx, uint64_t *data_dev, uint64_t count, int inverse, void *stream);

/*
 * AHE.Keygen (Fig. "SANNS linear-scan protocol", step 1): ternary secret s,
 * coefficient x = (lo mod 3) - 1 of ChaCha20 stream (seed, purpose 1,
 * object 0).  The key stays on the device.
 */
int sanns_keygen(sanns_ctx *ctx, uint64_t seed, sanns_sk **out, void *stream);
void sanns_sk_free(sanns_sk *sk);
/* Copy s (int8 [N]) and its NTT s_hat ([L][N]) to `any` memory; either
 * pointer may be NULL. */
int sanns_sk_export(const sanns_sk *sk, int8_t *s_any, uint64_t *s_hat_any, void *stream);

/*
 * Server-side encoding (Pi_ls step 3; Sec. 5.3 "g_i = sum_j p_{j+1}[i] x^j"):
 * position pos in [0, n) holds point perm[pos] (perm_dev NULL: identity,
 * n <= n_points).  Block k, dimension i is the polynomial whose coefficient x
 * is coordinate i of the point at position kN + x (zero past n), stored in
 * NTT form per prime and kept resident in HBM together with ||p||^2 per
 * position.  coords_dev: uint8 [n_points][d] row-major.  Synchronous; an
 * out-of-range perm entry returns SANNS_EINVAL.
 */
int sanns_encode_db(sanns_ctx *ctx, const uint8_t *coords_dev, uint64_t n_points,
                    const uint32_t *perm_dev, uint64_t n, sanns_db **out, void *stream);
void sanns_db_free(sanns_db *db);
/* Sharding (one shard of a database per GPU): the database encodes positions
 * pos0 .. pos0 + n - 1 of the whole permuted list (its perm argument being
 * that slice), so the mask of its local position x is drawn at global
 * position pos0 + x; outputs stay indexed locally.  pos0 must be a multiple
 * of N (shards are whole blocks).  Default 0. */
int sanns_db_set_position_base(sanns_db *db, uint64_t pos0);
/* n and K = ceil(n / N) of an encoded database. */
int sanns_db_info(const sanns_db *db, uint64_t *n, uint64_t *K);
/* Copy blocks [k0, k1) of the encoded plaintexts, layout [k][L][d][N], and
 * ||p||^2 of their (k1 - k0) N positions, to `any` memory (NULL skips). */
int sanns_db_export(const sanns_db *db, uint64_t k0, uint64_t k1, uint64_t *pt_any,
                    uint32_t *norms_any, void *stream);
/* The inverse of sanns_db_export over a whole database: a new encoded
 * database of n points (K = ceil(n / N) blocks) from its plaintexts pt_any
 * ([K][L][d][N], NTT form, canonical residues) and norms_any ([K N] uint32)
 * in `any` memory, for a server that encodes once (Pi_ls step 1, offline)
 * and loads the result later.  The context's current encoding setting is
 * recorded with it; position base 0.  The norms are stored reduced mod t
 * (the responses only ever use them mod t).  SANNS_EINVAL if a residue is
 * not below its prime (nothing is created).  Synchronous. */
int sanns_db_import(sanns_ctx *ctx, uint64_t n, const uint64_t *pt_any, const uint32_t *norms_any,
                    sanns_db **out, void *stream);

/*
 * AHE.Enc (Pi_ls step 2) of B queries, private-key BFV.  Coordinate i of
 * query b becomes the constant plaintext m = (t - 2 q[i]) mod t; per prime j
 *   a  = uniform mod q_j in NTT form, ChaCha20 stream (seed, 2,
 *        qid << 16 | j << 12 | i), slot s = draw s, value (hi 2^64 + lo) mod q_j;
 *   e  = centred binomial eta = 21 from stream (seed, 3, qid << 16 | i),
 *        draw x -> popcount(lo & (2^21-1)) - popcount((lo >> 21) & (2^21-1));
 *   c1 = a,   c0 = -a s_hat + NTT(e) + Delta_j m.
 * q_dev: uint8 [B][d]; qids_dev: uint64 [B] (qid < 2^48); ct_in_dev output
 * [B][d][2][L][N] in NTT form.
 */
int sanns_encrypt_query(sanns_ctx *ctx, const sanns_sk *sk, const uint8_t *q_dev, uint32_t B,
                        uint64_t seed, const uint64_t *qids_dev, uint64_t *ct_in_dev,
                        void *stream);

/*
 * Seeded query ciphertexts (the paper has no counterpart: its client sends
 * both components).  c1 = a of sanns_encrypt_query is the output of the
 * stream (seed, 2, qid << 16 | j << 12 | i), so a client may send c0 alone
 * with the seed and the query ids, halving the upload, and the server
 * rebuilds the ciphertext: ct_in_dev[b][i][0] = c0_dev[b][i] and
 * ct_in_dev[b][i][1] = a, bit-identical to sanns_encrypt_query's output for
 * the same (seed, qids).  c0_dev: [B][d][L][N] (component 0 of each
 * coordinate, NTT form); qids_dev: uint64 [B]; ct_in_dev output
 * [B][d][2][L][N].  The two buffers must not overlap; B <= 65535; SANNS_EINVAL
 * otherwise.  Asynchronous on stream.
 */
int sanns_expand_query(sanns_ctx *ctx, const uint64_t *c0_dev, uint32_t B, uint64_t seed,
                       const uint64_t *qids_dev, uint64_t *ct_in_dev, void *stream);

/*
 * The server's distance step (Pi_ls step 3) for B queries against one
 * encoded database:
 *   acc[b][k][c][j][s] = sum_i ct_in[b][i][c][j][s] pt[k][j][i][s]  mod q_j
 *   ct_out[b][k][c][j] = INTT_j(acc[b][k][c][j])
 *   ct_out[b][k][0][j][x] += Delta_j ((||p_pos||^2 + r_pos) mod t)
 * with pos = kN + x (padding included), r_pos uniform mod t from ChaCha20
 * stream (mask_seed, 4, qids[b]) draw pos, and the server's share
 *   srv_share[b][pos] = (t - r_pos) mod t for pos < n.
 * ct_in_dev [B][d][2][L][N] (NTT form), qids_dev uint64 [B], outputs
 * ct_out_dev [B][K][2][L][N] (coefficient form) and srv_share_dev uint32
 * [B][n].  The client's decryption plus ||q||^2 and the server's share add up
 * to ||q - p_pos||^2 mod t.
 */
int sanns_distances(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev, uint32_t B,
                    uint64_t mask_seed, const uint64_t *qids_dev, uint64_t *ct_out_dev,
                    uint32_t *srv_share_dev, void *stream);

/*
 * The two stages of sanns_distances, callable separately (same arguments,
 * same kernels, same launch configuration):
 *   sanns_distances_mac     acc[b][k][c][j][s] = sum_i ct_in pt mod q_j,
 *                           written to ct_out_dev in NTT form;
 *   sanns_distances_finish  in place on ct_out_dev: INTT, + Delta (||p||^2 +
 *                           r), and the server share.
 * sanns_distances(...) == sanns_distances_mac(...) then
 * sanns_distances_finish(...) on the same stream.
 */
int sanns_distances_mac(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev,
                        uint32_t B, uint64_t *ct_out_dev, void *stream);
int sanns_distances_finish(sanns_ctx *ctx, const sanns_db *db, uint32_t B, uint64_t mask_seed,
                           const uint64_t *qids_dev, uint64_t *ct_out_dev,
                           uint32_t *srv_share_dev, void *stream);

/*
 * Clustering protocol (Pi_cl steps 5-8; Algorithm 4, the distance loop over
 * the points of the retrieved clusters).  A clustering is C lists of point
 * indices in CSR form: cluster c holds members[offsets[c] .. offsets[c+1]).
 * sanns_clusters_create copies coords_dev (uint8 [n][d], any memory) and
 * members (uint32, any memory) into library-owned device memory and keeps
 * offsets_host (uint64 [C + 1]); a member index >= n returns SANNS_EINVAL.
 * Synchronous.
 */
int sanns_clusters_create(sanns_ctx *ctx, const uint8_t *coords_any, uint64_t n,
                          const uint64_t *offsets_host, const uint32_t *members_any, uint32_t C,
                          sanns_clusters **out, void *stream);
void sanns_clusters_free(sanns_clusters *cl);

/*
 * Host-only planning: for each query b with probe list probes_host[b][0..P)
 * (cluster ids, nearest first), n_out[b] = number of gathered points and
 * blocks_out[b] = ceil(n_out[b] / N) (blocks_out may be NULL).  The gathered
 * list of query b is the concatenation, in probe order, of the probed
 * clusters' member lists.
 */
int sanns_gather_plan(const sanns_clusters *cl, const uint32_t *probes_host, uint32_t B, uint32_t P,
                      uint64_t *n_out, uint64_t *blocks_out);

/*
 * Distances of B queries to their gathered lists in one persistent launch.
 * For query b the gathered list plays the role of the permuted database of
 * sanns_distances: position pos of the list is a point, blocks of N
 * positions are encoded, multiplied with ct_in[b], transformed back and
 * masked with r drawn from stream (mask_seed, 4, qids[b]) at pos.  The
 * context's circuit privacy and encoding apply as in sanns_distances, with
 * the list positions (from 0) as positions: each query's result is that of
 * sanns_distances on its gathered list as a database.
 * Outputs are concatenated query by query: ct_out_dev [sum_b blocks_b][2][L][N]
 * (in the context's response form), srv_share_dev uint32
 * [sum_b n_b], ids_dev uint32 [sum_b n_b] = the point index at each gathered
 * position (may be NULL).  Requires N <= 8192.  Uses a stream-ordered scratch
 * allocation of about sum_b blocks_b (d + 4 + 16 L S) N bytes (S dimension
 * slices, sized for about four units per SM) and synchronises the stream
 * once after uploading the plan.
 */
int sanns_distances_gather(sanns_ctx *ctx, const sanns_clusters *cl, const uint64_t *ct_in_dev,
                           uint32_t B, const uint32_t *probes_host, uint32_t P, uint64_t mask_seed,
                           const uint64_t *qids_dev, uint64_t *ct_out_dev, uint32_t *srv_share_dev,
                           uint32_t *ids_dev, void *stream);

/*
 * The same gather in two steps, for batches whose probes repeat and for CUDA
 * graph capture (the paper has no counterpart: its server handles one query
 * at a time).  sanns_gather_prepare plans the batch of probes_host (B x P,
 * host) and uploads the plan once (synchronous; the clusters must outlive
 * the batch).  sanns_distances_gather_prepared then computes exactly what
 * sanns_distances_gather computes for those probes, with the same output
 * layout (sizes from sanns_gather_plan); it only enqueues kernels and
 * stream-ordered scratch on stream, so it may be captured into a graph and
 * replayed (with new ciphertexts and query ids in the same buffers).  B in
 * 1..65535 and the other bounds of sanns_distances_gather; SANNS_EINVAL
 * otherwise.
 */
int sanns_gather_prepare(sanns_ctx *ctx, const sanns_clusters *cl, const uint32_t *probes_host,
                         uint32_t B, uint32_t P, sanns_gather_batch **out);
void sanns_gather_batch_free(sanns_gather_batch *batch);
int sanns_distances_gather_prepared(sanns_ctx *ctx, const sanns_gather_batch *batch,
                                    const uint64_t *ct_in_dev, uint64_t mask_seed,
                                    const uint64_t *qids_dev, uint64_t *ct_out_dev,
                                    uint32_t *srv_share_dev, uint32_t *ids_dev, void *stream);

/*
 * Launch variants of the MAC kernel (slots per lane, loads in flight, CTAs
 * per SM; one, "split_d_256x1", gives each work item a CTA whose warps split
 * the d dimensions, for launches with few items).  sanns_autotune_mac runs
 * every variant `reps` times on the given
 * inputs (writing ct_out_dev as sanns_distances_mac would), stores the
 * fastest in the context and returns its index (>= 0) or an error code;
 * ms_out (host, sanns_mac_variants() floats, may be NULL) receives the mean
 * time per launch.  Synchronous.  All variants compute identical results.
 */
int sanns_mac_variants(void);
const char *sanns_mac_variant_name(int variant);
int sanns_set_mac_variant(sanns_ctx *ctx, int variant);
/* SMs the MAC kernels' persistent grids spread over (0, the default: all),
 * for the per-query MAC and the batched tensor-core MAC alike (CTA pairs and
 * clusters take the largest whole number of pairs or clusters within it).
 * The per-query MAC is bound by HBM bandwidth, which fewer SMs can still
 * saturate, and the batched MAC by the board's power limit; the SMs left over
 * run other work launched on other streams at the same time, such as the
 * previous query's or batch's INTT + mask (sanns_distances_finish), whose
 * integer arithmetic then overlaps the next MAC.  Results never depend on
 * this value. */
int sanns_set_mac_sms(sanns_ctx *ctx, int sms);
int sanns_autotune_mac(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev, uint32_t B,
                       uint64_t *ct_out_dev, int reps, float *ms_out, void *stream);

/*
 * Batched path on the tensor cores (no counterpart in the paper, which
 * evaluates one query at a time): for B queries the per-slot work is the
 * dense contraction (2B x d) . (d x K) mod q_j, run as an exact fp16 GEMM
 * over balanced base-256 digits with fp32 accumulation (all partial sums are
 * integers below 2^24 for d <= 128).
 *   sanns_db_prepare_batched  builds the digit layout of the database once
 *                             ([L][N][K][8 ceil(d/8)] fp16, twice the size of
 *                             the encoded database) and its TMA descriptor.
 *                             Requires d <= 128.  Synchronous.
 *   sanns_distances_batched   same arguments and bit-identical results as
 *                             sanns_distances; B <= 4096.
 *   sanns_distances_batched_mac  its MAC stage alone (acc in NTT form).
 *   sanns_device_status       synchronises `stream` and returns
 *                             SANNS_ETIMEOUT (and clears it) if a bounded
 *                             device-side wait of a batched launch gave up.
 */
int sanns_db_prepare_batched(sanns_ctx *ctx, sanns_db *db, void *stream);
int sanns_distances_batched(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev,
                            uint32_t B, uint64_t mask_seed, const uint64_t *qids_dev,
                            uint64_t *ct_out_dev, uint32_t *srv_share_dev, void *stream);
int sanns_distances_batched_mac(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev,
                                uint32_t B, uint64_t *ct_out_dev, void *stream);
int sanns_device_status(sanns_ctx *ctx, void *stream);
/*
 * Self-test of the failure path of the bounded device-side waits (no
 * counterpart in the paper): one thread waits, with the batched kernel's own
 * bounded-wait routine, on a shared-memory barrier that nothing completes;
 * after limit_ms (1 .. 1000) the wait gives up, raises the context's device
 * error word and the kernel returns, so the next sanns_device_status returns
 * SANNS_ETIMEOUT (and clears it) and the context stays usable.  It faults
 * nothing and always ends.  Asynchronous on stream.
 */
int sanns_selftest_wait_timeout(sanns_ctx *ctx, uint32_t limit_ms, void *stream);
/*
 * Measured dense tensor-core rates of the current GPU (no counterpart in the
 * paper; the denominators of the batched path's roofline).  Runs three
 * throughput probes on every SM and writes, to rates_host[0..2]:
 *   [0] tcgen05.mma kind::f16, M128 N256 K16, fp16 in, fp32 out (TFLOP/s);
 *       the instruction family of the batched MAC;
 *   [1] legacy mma.sync m16n8k16, fp16 in, fp32 out (TFLOP/s);
 *   [2] legacy mma.sync m16n8k32, s8 in, s32 out (TOP/s), the only INT8
 *       tensor instruction on sm_103a: ptxas rejects tcgen05.mma kind::i8
 *       for that target.
 * Synchronous, about 10 ms of GPU time.  SANNS_ETIMEOUT if the probe's
 * bounded completion wait gave up (nothing is written then).
 */
int sanns_measure_mma_rates(sanns_ctx *ctx, double *rates_host, void *stream);
/*
 * Measured integer-pipe ceiling of the transforms (no counterpart in the
 * paper; the denominator of the INTT and gather rooflines): radix-2
 * butterflies per second on every SM, values in registers, the context's
 * first prime, written to rates_host[0] (inverse, Gentleman-Sande, the fused
 * INTT's lazy arithmetic) and rates_host[1] (forward, Cooley-Tukey).
 * Synchronous, a few milliseconds of GPU time.
 */
int sanns_measure_int_rates(sanns_ctx *ctx, double *rates_host, void *stream);
/*
 * Device memory a distance call allocates for itself, beyond the caller's
 * buffers (no counterpart in the paper; for admission control by device
 * memory): *bytes = the stream-ordered scratch of one sanns_distances call
 * (batched = 0: none, the per-query path writes the caller's buffers only)
 * or one sanns_distances_batched call with B queries under the context's
 * current tuning (batched != 0: the query multiples of one slot range,
 * bounded by the scratch cap of sanns_batched_tune).  It is freed on the
 * call's stream when the call's work is done.
 */
int sanns_distances_scratch_bytes(const sanns_ctx *ctx, uint32_t B, int batched, uint64_t *bytes);
/* Tuning of the batched kernel: back-off sleep (ns, <= 100000) of the TMA
 * thread, the MMA thread, the digit producers and the epilogue when their
 * barrier is not ready yet; how many of its own work units ahead each CTA
 * prefetches the database-digit and query tiles into L2 (0 = no prefetch,
 * <= 8; default 0); the cap (MiB, default 4096) on the stream-ordered
 * scratch that holds the query multiples of one range of slots (a smaller cap
 * means more, shorter launches; at least one slot's worth is always used);
 * and the tile shape, two bits: bit 0 clear = 128 database blocks x 256 query
 * rows per SM, set = 256 x 256 per pair of SMs (cluster of two CTAs sharing
 * one MMA); bit 1 clear = producer warps turn byte-interleaved query
 * multiples into fp16 digit rows in shared memory, set = a pre-kernel writes
 * the fp16 digit rows to the scratch once per slot range (twice the scratch
 * per slot) and they arrive by TMA like the database tile; 4 and 5 = the
 * one-SM, TMA-fed tile run by clusters of 2 or 4 CTAs that take consecutive
 * database tiles of one slot and query tile and share the query tile by
 * multicast (each CTA loads a 1/2 or 1/4 of it for all); 6 and 7 = the
 * one-SM, TMA-fed tile with four consecutive slots per CTA, whose epilogue
 * holds three slots in registers and writes each output's four slots as one
 * 32-byte store (a whole sector), alone (6) or in clusters of 2 sharing the
 * query tile (7; as 6 when the number of 128-block database tiles is odd);
 * 8 = the four-slot epilogue on pairs of SMs (256 database blocks x 256
 * query rows per pair, each CTA loading its 128 blocks and half of the query
 * tile by TMA).
 * Defaults: tile 7, no L2 prefetch (the fastest on the n = 10^7, d = 96,
 * 64-query workload).
 * Results never depend on these values.  Returns SANNS_EINVAL for
 * out-of-range values. */
int sanns_batched_tune(sanns_ctx *ctx, uint32_t tma_ns, uint32_t mma_ns, uint32_t producer_ns,
                       uint32_t epilogue_ns, uint32_t prefetch_units, uint32_t scratch_mib,
                       uint32_t tile);
/* Autotuner of the batched MAC: times the eighteen configurations cfg = 2 tile +
 * prefetch_units (tile 0..8, L2 prefetch 0 or 1 unit ahead) `reps` times
 * each on the given inputs (writing ct_out_dev as sanns_distances_batched_mac
 * would), keeps the fastest in the context and returns its index (>= 0) or an
 * error code; ms_out (host, 18 floats, may be NULL) receives the mean time per
 * launch.  Synchronous.  Every configuration computes identical results. */
int sanns_autotune_batched(sanns_ctx *ctx, const sanns_db *db, const uint64_t *ct_in_dev, uint32_t B,
                           uint64_t *ct_out_dev, int reps, float *ms_out, void *stream);

/*
 * Plaintext encoding of the database (Sec. 5.3 packs N points per
 * plaintext; Sec. 7.1 picks t; SEAL's batching puts values in the CRT slots
 * mod t when t = 1 mod 2N).
 *   0 (default)  coefficient encoding: point x of a block is coefficient x.
 *   1            slot encoding: point x of a block is CRT slot x mod t.  The
 *                plaintext of a coordinate row is the inverse negacyclic
 *                transform mod t (psi_t = the smallest primitive 2N-th root
 *                of unity mod t) of the row, with coefficients in [0, t); the
 *                norms are encoded the same way; the server's mask is a
 *                polynomial R whose coefficients are drawn as in coefficient
 *                encoding (padding included), and its share of slot x is
 *                t - NTT_t(R)[x]; the client's share is NTT_t(m)[x] +
 *                ||q||^2.  Shares are identical in meaning to coefficient
 *                encoding: they add up to ||q - p||^2 mod t.
 * A database keeps the encoding the context had when it was encoded; the
 * distance calls reject a database whose encoding differs from the context's.
 * Slot encoding combines with NTT-form responses (the NTT of the slot-encoded
 * coefficient response) and with circuit privacy.
 * sanns_decrypt_shares (and its no-allocation variant) decode in the
 * context's encoding.  SANNS_EINVAL for slots when t != 1 mod 2N.
 */
int sanns_set_encoding(sanns_ctx *ctx, int slots);

/*
 * Response form.  0 (default): coefficient form, as the paper's protocol
 * returns (the server transforms every response polynomial back).  1: NTT
 * form, the NTT (per prime, the same negacyclic transform as the queries') of
 * the coefficient-form response, bit for bit: the server skips both inverse
 * transforms and adds NTT(Delta (||p||^2 + r)) to c0 (L forward transforms per
 * block instead of 2L inverse ones), and sanns_decrypt_shares on a context in
 * this form takes one inverse transform per block and prime.  Both sides of a
 * protocol run must use the same form.  The gather path answers in
 * coefficient form only and rejects calls while form 1 is set.
 */
int sanns_set_response_form(sanns_ctx *ctx, int form);

/*
 * Response modulus (an option beyond the paper, whose server sends the
 * responses at the full modulus Q = q_0 ... q_{L-1}).  primes = L (default):
 * as the paper.  primes = 1: after the epilogue the server switches every
 * coefficient-form response down to q_0, the standard BFV modulus switch
 * c -> round(q_0 c / Q) mod q_0 of each coefficient c in [0, Q), computed in
 * RNS (Garner digits of the dropped primes, exact), so a response costs 1/L
 * of the bytes.  After the switch the phase noise is (q_0 / Q) e plus at
 * most (N + 1) / 2 of rounding; with e up to the largest circuit-privacy
 * flooding (Q / (4t)) it stays below q_0 / (2t), so decryption is unchanged,
 * whenever q_0 > 2t (N + 5) -- the call returns SANNS_EINVAL otherwise.
 *   - sanns_distances / sanns_distances_batched then leave the switched
 *     response in the j = 0 rows of ct_out_dev ([B][K][2][L][N], rows of N
 *     words at a pitch of L N); the other rows are scratch.
 *     sanns_copy_responses gathers them compact.
 *   - sanns_decrypt_shares(_noalloc) on a context with primes = 1 takes the
 *     compact switched responses, [B][K][2][N], and decrypts modulo q_0.
 *   - The clustering gather does the same to each work item's response
 *     ([W][2][L][N]: its j = 0 rows; sanns_copy_responses with B = 1,
 *     K = W gathers them).
 *   - Not with NTT-form responses (SANNS_EINVAL either way round).
 * Both sides of a protocol run must use the same setting.
 */
int sanns_set_response_primes(sanns_ctx *ctx, uint32_t primes);

/*
 * Copies the responses of B queries over K blocks from ct_out_dev (as a
 * distance call left them) to dst, compact: [B][K][2][R][N] with R the
 * response primes (L: the whole buffer; 1: the j = 0 rows).  dst may be
 * device memory or pinned host memory (the download of a response).
 * Asynchronous on stream.
 */
int sanns_copy_responses(const sanns_ctx *ctx, const uint64_t *ct_out_dev, uint32_t B, uint64_t K,
                         uint64_t *dst, void *stream);

/*
 * Plaintext meaning of the selection step (Sec. 4, Algorithms 1 and 2; the
 * paper evaluates it inside garbled circuits, which this library does not):
 * for every query b the k smallest reconstructed distances
 * ((cli_dev[b][x] + srv_dev[b][x]) mod t) >> shift over positions x < n
 * (shift <= 31: Algorithm 4 truncates distances by 2^r_c or 2^r_p before
 * selecting).
 *   bins = 0:  exact, the k smallest (distance, position) pairs in that order,
 *              which is the result Algorithm 1 (NaiveTopk) produces.
 *   bins = l:  Algorithm 2 (ApproxTopk): position x falls in bin
 *              floor(x l / n); the minimum of every bin (the earlier position
 *              on ties), then the k smallest of the l minima.
 * Output (device, caller-owned): dist_dev [B][k] u32 ascending, pos_dev
 * [B][k] u64 positions (in the server's permuted order).  Needs 1 <= k <=
 * 1024, B <= 65535, k <= n < 2^32 and, for l > 0, k <= l <= n; SANNS_EINVAL
 * otherwise.  k <= 32 keeps per-thread register lists; larger k sorts chunks
 * of 4096 keys in shared memory.
 * Asynchronous on stream (stream-ordered scratch).
 */
int sanns_topk(sanns_ctx *ctx, const uint32_t *cli_dev, const uint32_t *srv_dev, uint32_t B, uint64_t n,
               uint32_t k, uint64_t bins, uint32_t shift, uint32_t *dist_dev, uint64_t *pos_dev,
               void *stream);

/*
 * The same selection over B ragged lists (Algorithm 4: the points gathered
 * for each query, the centres of one group): list b is positions x <
 * len[b] of cli_dev + cli_off[b] and srv_dev + srv_off[b]; positions in the
 * output count from the list's start.  List b selects k_b = k_seg[b]
 * winners (k_seg NULL: k for every list; 1 <= k_b <= k).  With bins = 0 every
 * list is exact; otherwise list b is ApproxTopk over l_b = bins_seg[b]
 * (bins_seg NULL: bins; k_b <= l_b <= bins) bins, of which it uses
 * min(l_b, len[b]) (every position its own bin, i.e. exact, when len[b] <=
 * l_b).  Outputs are [B][k]: list b's k_b winners, then fill entries with
 * dist 2^32 - 1 and pos 2^64 - 1 (also where a list holds fewer than k_b
 * elements; the uniform call never produces them).  cli_off, srv_off, len,
 * k_seg and bins_seg are HOST arrays of B entries, read before the call
 * returns; the device shares must hold every listed element.  Needs 1 <= k <=
 * 1024, B <= 65535, len[b] < 2^32, bins = 0 or bins >= k_b, shift <= 31;
 * SANNS_EINVAL otherwise.  Stream-ordered scratch; the host arrays are copied
 * (pageable) on stream.
 */
int sanns_topk_segments(sanns_ctx *ctx, const uint32_t *cli_dev, const uint32_t *srv_dev, uint32_t B,
                        const uint64_t *cli_off, const uint64_t *srv_off, const uint64_t *len,
                        const uint32_t *k_seg, const uint64_t *bins_seg, uint32_t k,
                        uint64_t bins, uint32_t shift, uint32_t *dist_dev, uint64_t *pos_dev, void *stream);

/*
 * Circuit privacy (Sec. 2.3, "Additive Homomorphic Encryption": the AHE scheme
 * must not reveal the server's operations beyond the decrypted message; the
 * paper obtains this by noise flooding, with 108 bits of statistical circuit
 * privacy at its parameters, Sec. 7.1).  Private-key BFV leaves the server
 * unable to re-randomise c1, so the client also publishes a public key and
 * the server adds a fresh encryption of zero (pk0 u + e1, pk1 u + e2) to every
 * response block, e1 being the flooding term, uniform in [-2^F, 2^F).
 *   sanns_public_key      client: pk_dev (device, [2][L][N] u64, NTT form,
 *                         caller-owned) = (-a s + e, a), a drawn in NTT form
 *                         from stream (seed, 5, prime j), e centred binomial
 *                         (eta = 21) from (seed, 6, 0).  Asynchronous on stream.
 *   sanns_set_circuit_privacy  server: copies the key into the context (the
 *                         caller's buffer may be freed afterwards) and sets F;
 *                         every later sanns_distances / _finish /
 *                         _batched on this context then adds, per query b and
 *                         global position x (streams keyed by mask_seed and
 *                         qids[b]): u ternary (purpose 7), pk * NTT(u) before
 *                         the inverse transform; e1 = low F + 1 bits of two
 *                         128-bit draws (purposes 9, 10) minus 2^F to c0 and
 *                         e2 centred binomial (purpose 8) to c1 after it.
 *                         pk_dev = NULL turns it off.  F above
 *                         sanns_circuit_privacy_max_flood_bits (2^F <= Delta /
 *                         4, so decryption stays correct) returns SANNS_EINVAL.
 *                         Synchronous.
 */
int sanns_public_key(sanns_ctx *ctx, const sanns_sk *sk, uint64_t seed, uint64_t *pk_dev, void *stream);
int sanns_circuit_privacy_max_flood_bits(const sanns_ctx *ctx);
int sanns_set_circuit_privacy(sanns_ctx *ctx, const uint64_t *pk_dev, uint32_t flood_bits, void *stream);

/*
 * Client decryption (Pi_ls step 4) plus its local term: per query b and
 * position pos < n, m = round(t (c0 + c1 s mod Q) / Q) mod t (CRT over the L
 * primes), cli_share[b][pos] = (m + ||q_b||^2) mod t.  ct_out_dev
 * [B][K][2][L][N] with K = ceil(n / N); q_dev uint8 [B][d]; cli_share_dev
 * uint32 [B][n].  Uses a stream-ordered scratch allocation of B K L N words.
 * With sanns_set_response_primes(ctx, 1): ct_out_dev is [B][K][2][N] modulo
 * q_0 (sanns_copy_responses' compact form), Q is q_0, and the scratch is
 * B K N words.
 */
int sanns_decrypt_shares(sanns_ctx *ctx, const sanns_sk *sk, const uint64_t *ct_out_dev,
                         uint32_t B, uint64_t n, const uint8_t *q_dev, uint32_t *cli_share_dev,
                         void *stream);

/*
 * sanns_decrypt_shares_noalloc -- the paper has no counterpart to this entry
 * point; it exists for callers that cannot allocate device memory while they
 * run: code being captured into a CUDA graph, real-time loops that may not
 * call cudaMalloc (it can synchronise the device and has unbounded latency),
 * and processes held to a fixed device-memory budget.  Same arguments,
 * kernels and results as sanns_decrypt_shares, but it allocates nothing: its
 * scratch is a file-scope device array of sanns_decrypt_noalloc_max_words()
 * = 4,194,304 uint64 words (32 MiB), which every GPU that loads the library
 * holds until the process exits.
 *   - B * ceil(n / N) * L * N must not exceed that maximum; larger requests
 *     return SANNS_EINVAL before anything is launched (one N = 8192, L = 3
 *     query fits up to n = 1,392,640 points).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: resetting the device (cudaDeviceReset) and calling again is
 *     not supported.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call writes every word it later reads, so nothing is cleared, but
 *     calls that overlap on the GPU (different streams, no ordering between
 *     them) race on the array: order them on one stream or with events.
 */
int sanns_decrypt_shares_noalloc(sanns_ctx *ctx, const sanns_sk *sk, const uint64_t *ct_out_dev,
                                 uint32_t B, uint64_t n, const uint8_t *q_dev,
                                 uint32_t *cli_share_dev, void *stream);
uint64_t sanns_decrypt_noalloc_max_words(void);

/* Number of multiprocessors the persistent kernels size their grids by. */
int sanns_device_sms(void);

#ifdef __cplusplus
}
#endif
#endif /* SANNS_H_ */
