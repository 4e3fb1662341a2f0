/*
 * sanns_oracle.c -- plain, slow CPU oracle for the encrypted-distance path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline and reference legs of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: every routine
 * below is written out directly from its definition, with no lazy reduction,
 * no blocking and no fusion.
 *
 * What it follows (SANNS, arxiv 1904.02033):
 *   - Sec. 5.3 "Distance Computation via AHE": the client encrypts each query
 *     coordinate as a constant polynomial f_i, the server encodes coordinate i
 *     of N points as g_i = sum_j p_{j+1}[i] x^j and computes sum_i f_i g_i,
 *     masks it with a random polynomial and returns it.
 *   - Fig. "SANNS linear-scan protocol" (Pi_ls), steps 2-4: Enc of the d
 *     coordinates, f_k = sum_i CMult(c_i, p_ik) + r[kN:(k+1)N], decryption.
 *   - Sec. 2.3 (AHE): BFV [FV12]; R_t = Z_t[x]/(x^N + 1).
 * The BFV conventions the paper leaves to SEAL (NTT order, RNG, sampling,
 * Delta) are fixed here as readings of the paper; each function states the
 * one it implements.
 *
 * Arithmetic: all residues are canonical uint64 in [0, q); every product is a
 * 128-bit product reduced with the C '%' operator.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* modular arithmetic, written out                                      */
/* ------------------------------------------------------------------ */
static uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q)
{
    u128 s = (u128)a + b;
    return (uint64_t)(s % q);
}

static uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q)
{
    /* a, b in [0, q) */
    return a >= b ? a - b : (uint64_t)((u128)a + q - b);
}

static uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * b) % q);
}

static uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mul_mod(r, a, q);
        a = mul_mod(a, a, q);
        e >>= 1;
    }
    return r;
}

static uint32_t bit_reverse(uint32_t x, int bits)
{
    uint32_t r = 0;
    for (int b = 0; b < bits; b++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

static int log2_exact(uint32_t n)
{
    int l = 0;
    while ((1u << l) < n) l++;
    return l;
}

/* ------------------------------------------------------------------ */
/* NTT over Z_q[x]/(x^N + 1)                                             */
/* ------------------------------------------------------------------ */
/*
 * Products in the BFV ring R_q = Z_q[x]/(x^N + 1) (Sec. 2.3, Sec. 5.3).  The
 * paper leaves the multiplication algorithm to SEAL; this is the textbook
 * negacyclic number-theoretic transform.
 */
/*
 * Twiddle tables: fwd[m] = psi^brv(m), inv[m] = psi^-brv(m), m in [0, N),
 * brv over log2(N) bits.
 */
void oracle_ntt_tables(uint32_t N, uint64_t q, uint64_t psi,
                       uint64_t *fwd, uint64_t *inv)
{
    int logn = log2_exact(N);
    uint64_t psi_inv = pow_mod(psi, q - 2, q);
    for (uint32_t m = 0; m < N; m++) {
        uint32_t e = bit_reverse(m, logn);
        fwd[m] = pow_mod(psi, e, q);
        inv[m] = pow_mod(psi_inv, e, q);
    }
}

/*
 * Forward negacyclic NTT, in place: the textbook iterative Cooley-Tukey
 * transform without a reordering pass.  Its output in position s is the
 * evaluation a(psi^(2 brv(s) + 1)) mod q (the tests check this against the
 * O(N^2) definition).
 */
void oracle_ntt(uint64_t *a, uint32_t N, uint64_t q, const uint64_t *fwd)
{
    uint32_t t = N;
    for (uint32_t m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (uint32_t i = 0; i < m; i++) {
            uint64_t w = fwd[m + i];
            uint32_t j1 = 2 * i * t;
            for (uint32_t j = j1; j < j1 + t; j++) {
                uint64_t u = a[j];
                uint64_t v = mul_mod(a[j + t], w, q);
                a[j] = add_mod(u, v, q);
                a[j + t] = sub_mod(u, v, q);
            }
        }
    }
}

/*
 * Inverse of oracle_ntt: Gentleman-Sande butterflies in the reverse stage
 * order, then multiplication by N^-1 mod q.
 */
void oracle_intt(uint64_t *a, uint32_t N, uint64_t q, const uint64_t *inv)
{
    uint32_t t = 1;
    for (uint32_t m = N; m > 1; m >>= 1) {
        uint32_t h = m >> 1;
        for (uint32_t i = 0; i < h; i++) {
            uint64_t w = inv[h + i];
            uint32_t j1 = 2 * i * t;
            for (uint32_t j = j1; j < j1 + t; j++) {
                uint64_t u = a[j];
                uint64_t v = a[j + t];
                a[j] = add_mod(u, v, q);
                a[j + t] = mul_mod(sub_mod(u, v, q), w, q);
            }
        }
        t <<= 1;
    }
    uint64_t n_inv = pow_mod(N, q - 2, q);
    for (uint32_t j = 0; j < N; j++) a[j] = mul_mod(a[j], n_inv, q);
}

/* ------------------------------------------------------------------ */
/* ChaCha20 block function (RFC 8439, its section 2.3)                  */
/* ------------------------------------------------------------------ */
/*
 * The randomness of keygen, encryption, the server's masks and circuit
 * privacy (Sec. 2.3, Sec. 5.3).  The paper leaves its source to SEAL; every
 * draw here comes from a ChaCha20 stream.
 */
static uint32_t rotl32(uint32_t x, int n) { return (x << n) | (x >> (32 - n)); }

static void quarter_round(uint32_t *s, int a, int b, int c, int d)
{
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}

void oracle_chacha20_block(const uint32_t key[8], uint32_t counter,
                           const uint32_t nonce[3], uint32_t out[16])
{
    uint32_t init[16];
    init[0] = 0x61707865u; init[1] = 0x3320646eu;
    init[2] = 0x79622d32u; init[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) init[4 + i] = key[i];
    init[12] = counter;
    init[13] = nonce[0]; init[14] = nonce[1]; init[15] = nonce[2];
    uint32_t w[16];
    memcpy(w, init, sizeof(w));
    for (int r = 0; r < 10; r++) {
        quarter_round(w, 0, 4, 8, 12);
        quarter_round(w, 1, 5, 9, 13);
        quarter_round(w, 2, 6, 10, 14);
        quarter_round(w, 3, 7, 11, 15);
        quarter_round(w, 0, 5, 10, 15);
        quarter_round(w, 1, 6, 11, 12);
        quarter_round(w, 2, 7, 8, 13);
        quarter_round(w, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = w[i] + init[i];
}

/*
 * Draw the 128 random bits of coefficient c from stream (seed, purpose,
 * object): key = seed as two little-endian words, rest zero; nonce = (purpose,
 * object low word, object high word); block counter = c / 4; the draw is the
 * four words 4 (c mod 4) .. 4 (c mod 4) + 3 of that block, read as
 * lo = w0 | w1 << 32, hi = w2 | w3 << 32.
 */
enum { PURPOSE_SK = 1, PURPOSE_A = 2, PURPOSE_E = 3, PURPOSE_MASK = 4,
       /* circuit privacy: public key (client), re-randomisation and flooding (server) */
       PURPOSE_A_PK = 5, PURPOSE_E_PK = 6, PURPOSE_U = 7, PURPOSE_E2 = 8,
       PURPOSE_FLOOD_LO = 9, PURPOSE_FLOOD_HI = 10 };

static void draw128(uint64_t seed, uint32_t purpose, uint64_t object,
                    uint64_t c, uint64_t *lo, uint64_t *hi)
{
    uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
    uint32_t nonce[3] = {purpose, (uint32_t)object, (uint32_t)(object >> 32)};
    uint32_t blk[16];
    oracle_chacha20_block(key, (uint32_t)(c / 4), nonce, blk);
    const uint32_t *w = blk + 4 * (c % 4);
    *lo = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    *hi = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
}

void oracle_draw128(uint64_t seed, uint32_t purpose, uint64_t object,
                    uint64_t c, uint64_t out[2])
{
    draw128(seed, purpose, object, c, &out[0], &out[1]);
}

/* samplers */
static int ternary_of(uint64_t lo) { return (int)(lo % 3) - 1; }

static int cbd21_of(uint64_t lo)
{
    uint64_t m = (1ull << 21) - 1;
    return __builtin_popcountll(lo & m) - __builtin_popcountll((lo >> 21) & m);
}

static uint64_t uniform_of(uint64_t lo, uint64_t hi, uint64_t m)
{
    u128 v = ((u128)hi << 64) | lo;
    return (uint64_t)(v % m);
}

/* signed small integer -> residue mod q */
static uint64_t lift(int64_t v, uint64_t q)
{
    return v >= 0 ? (uint64_t)v % q : q - ((uint64_t)(-v) % q);
}

/* ------------------------------------------------------------------ */
/* the protocol steps                                                   */
/* ------------------------------------------------------------------ */
/*
 * Parameter block passed from Python (oracle/params.py computes every value
 * with exact big integers):
 *   q[L], fwd[L][N], inv[L][N] (twiddles from oracle_ntt_tables), t,
 *   delta[L] = floor(Q / t) mod q_j.
 */
typedef struct {
    uint32_t N, L, d, pad;
    uint64_t t;
    const uint64_t *q;
    const uint64_t *fwd;
    const uint64_t *inv;
    const uint64_t *delta;
} oracle_params;

/*
 * AHE.Keygen (Pi_ls step 1): ternary secret s, coefficient x drawn from
 * stream (seed, SK, 0) as (lo mod 3) - 1.  Returns s (int8, [N]) and its NTT
 * per prime s_hat [L][N].
 */
void oracle_keygen(const oracle_params *P, uint64_t seed, int8_t *s,
                   uint64_t *s_hat)
{
    uint32_t N = P->N;
    for (uint32_t x = 0; x < N; x++) {
        uint64_t lo, hi;
        draw128(seed, PURPOSE_SK, 0, x, &lo, &hi);
        s[x] = (int8_t)ternary_of(lo);
    }
    for (uint32_t j = 0; j < P->L; j++) {
        uint64_t *sh = s_hat + (size_t)j * N;
        for (uint32_t x = 0; x < N; x++) sh[x] = lift(s[x], P->q[j]);
        oracle_ntt(sh, N, P->q[j], P->fwd + (size_t)j * N);
    }
}

/*
 * AHE.Enc of one query (Pi_ls step 2), private-key BFV.  For coordinate i the
 * plaintext is the constant polynomial m_i = (t - 2 q[i]) mod t (the factor
 * -2 of the distance expansion sits on the client).  Per prime j:
 *   a     uniform mod q_j, drawn directly in NTT form from stream
 *         (seed, A, qid << 16 | j << 12 | i), slot s = coefficient s;
 *   e     centred binomial (eta = 21) from stream (seed, E, qid << 16 | i),
 *         one integer polynomial lifted into every prime, then NTT;
 *   c1    = a,  c0 = -a * s_hat + e_hat + Delta_j * m_i  (slot-wise).
 * A constant polynomial's NTT is the same constant in every slot, so
 * Delta_j * m_i is added to every slot.
 * Output ct[i][c][j][s], NTT form, c = 0, 1.
 */
void oracle_encrypt(const oracle_params *P, const uint64_t *s_hat,
                    const uint8_t *qv, uint64_t seed, uint64_t qid,
                    uint64_t *ct)
{
    uint32_t N = P->N, L = P->L, d = P->d;
    uint64_t t = P->t;
    uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * N);
    int64_t *ei = (int64_t *)malloc(sizeof(int64_t) * N);
    for (uint32_t i = 0; i < d; i++) {
        uint64_t m = (t - (2 * (uint64_t)qv[i]) % t) % t;
        for (uint32_t x = 0; x < N; x++) {
            uint64_t lo, hi;
            draw128(seed, PURPOSE_E, (qid << 16) | i, x, &lo, &hi);
            ei[x] = cbd21_of(lo);
        }
        for (uint32_t j = 0; j < L; j++) {
            uint64_t q = P->q[j];
            for (uint32_t x = 0; x < N; x++) e[x] = lift(ei[x], q);
            oracle_ntt(e, N, q, P->fwd + (size_t)j * N);
            uint64_t dm = mul_mod(P->delta[j], m, q);
            uint64_t *c0 = ct + (((size_t)i * 2 + 0) * L + j) * N;
            uint64_t *c1 = ct + (((size_t)i * 2 + 1) * L + j) * N;
            const uint64_t *sh = s_hat + (size_t)j * N;
            uint64_t obj = (qid << 16) | ((uint64_t)j << 12) | i;
            for (uint32_t s = 0; s < N; s++) {
                uint64_t lo, hi;
                draw128(seed, PURPOSE_A, obj, s, &lo, &hi);
                uint64_t a = uniform_of(lo, hi, q);
                c1[s] = a;
                uint64_t v = sub_mod(0, mul_mod(a, sh[s], q), q);
                v = add_mod(v, e[s], q);
                v = add_mod(v, dm, q);
                c0[s] = v;
            }
        }
    }
    free(e);
    free(ei);
}

/*
 * Server-side encoding of the database (Pi_ls step 3, Sec. 5.3): block k,
 * dimension i, prime j holds the polynomial whose coefficient x is
 * coordinate i of the point at permuted position kN + x (zero past n), in
 * NTT form.  perm[pos] is the original index of the point at position pos.
 * Only blocks [k0, k1) are produced, pt laid out [k - k0][j][i][s].
 * norms[pos - k0 N] = ||p||^2 for pos < n, else 0.
 */
void oracle_encode_db(const oracle_params *P, const uint8_t *coords,
                      const uint32_t *perm, uint64_t n, uint64_t k0,
                      uint64_t k1, uint64_t *pt, uint32_t *norms)
{
    uint32_t N = P->N, L = P->L, d = P->d;
    for (uint64_t k = k0; k < k1; k++) {
        for (uint32_t x = 0; x < N; x++) {
            uint64_t pos = k * N + x;
            uint32_t nrm = 0;
            if (pos < n) {
                const uint8_t *p = coords + (size_t)perm[pos] * d;
                for (uint32_t i = 0; i < d; i++) nrm += (uint32_t)p[i] * p[i];
            }
            norms[(k - k0) * N + x] = nrm;
        }
        for (uint32_t j = 0; j < L; j++) {
            for (uint32_t i = 0; i < d; i++) {
                uint64_t *poly = pt + ((((k - k0) * L) + j) * d + i) * N;
                for (uint32_t x = 0; x < N; x++) {
                    uint64_t pos = k * N + x;
                    poly[x] = pos < n ? coords[(size_t)perm[pos] * d + i] : 0;
                }
                oracle_ntt(poly, N, P->q[j], P->fwd + (size_t)j * N);
            }
        }
    }
}

/*
 * ct x pt multiply-accumulate (Pi_ls step 3, sum_i CMult(c_i, p_ik)): in the
 * NTT domain a ciphertext-plaintext product is slot-wise, so for every block
 * k of [0, nk), poly c, prime j and slot s
 *   acc[k][c][j][s] = sum_i ct[i][c][j][s] * pt[k][j][i][s]  mod q_j.
 */
void oracle_mac(const oracle_params *P, const uint64_t *ct, const uint64_t *pt,
                uint64_t nk, uint64_t *acc)
{
    uint32_t N = P->N, L = P->L, d = P->d;
    for (uint64_t k = 0; k < nk; k++)
        for (uint32_t c = 0; c < 2; c++)
            for (uint32_t j = 0; j < L; j++) {
                uint64_t q = P->q[j];
                uint64_t *out = acc + ((k * 2 + c) * L + j) * N;
                for (uint32_t s = 0; s < N; s++) {
                    uint64_t sum = 0;
                    for (uint32_t i = 0; i < d; i++) {
                        uint64_t cv = ct[(((size_t)i * 2 + c) * L + j) * N + s];
                        uint64_t pv = pt[((k * L + j) * d + i) * N + s];
                        sum = add_mod(sum, mul_mod(cv, pv, q), q);
                    }
                    out[s] = sum;
                }
            }
}

/*
 * Back to coefficient form and mask (Pi_ls step 3, "+ r[kN:(k+1)N]").  For
 * blocks k in [k0, k1) (acc and out indexed from k0):
 *   out[k][c][j] = INTT_j(acc[k][c][j]);
 *   for c = 0 and every position pos = kN + x (padding included):
 *     r   = uniform mod t from stream (mask_seed, MASK, qid), coefficient pos;
 *     out += Delta_j * ((||p_pos||^2 + r) mod t)  mod q_j;
 *   srv_share[pos] = (t - r) mod t for pos < n.
 * Adding Delta * ||p||^2 moves the server's local term of the distance
 * expansion into the ciphertext, so the shares reconstruct ||q - p||^2.
 */
void oracle_intt_mask(const oracle_params *P, const uint64_t *acc,
                      const uint32_t *norms, uint64_t n, uint64_t k0,
                      uint64_t k1, uint64_t mask_seed, uint64_t qid,
                      uint64_t *out, uint32_t *srv_share)
{
    uint32_t N = P->N, L = P->L;
    uint64_t t = P->t;
    for (uint64_t k = k0; k < k1; k++) {
        for (uint32_t c = 0; c < 2; c++)
            for (uint32_t j = 0; j < L; j++) {
                size_t off = (((k - k0) * 2 + c) * L + j) * N;
                memcpy(out + off, acc + off, sizeof(uint64_t) * N);
                oracle_intt(out + off, N, P->q[j], P->inv + (size_t)j * N);
            }
        for (uint32_t x = 0; x < N; x++) {
            uint64_t pos = k * N + x;
            uint64_t lo, hi;
            draw128(mask_seed, PURPOSE_MASK, qid, pos, &lo, &hi);
            uint64_t r = uniform_of(lo, hi, t);
            uint64_t v = ((uint64_t)norms[(k - k0) * N + x] + r) % t;
            for (uint32_t j = 0; j < L; j++) {
                uint64_t q = P->q[j];
                size_t off = (((k - k0) * 2 + 0) * L + j) * N + x;
                out[off] = add_mod(out[off], mul_mod(P->delta[j], v, q), q);
            }
            if (pos < n) srv_share[pos - k0 * N] = (uint32_t)((t - r) % t);
        }
    }
}

/* ------------------------------------------------------------------ */
/* circuit privacy                                                      */
/* ------------------------------------------------------------------ */
/*
 * The paper asks the AHE scheme for circuit privacy and obtains it by noise
 * flooding (Sec. 2.3, "Additive Homomorphic Encryption"; 108 bits of
 * statistical circuit privacy with its parameters, Sec. 7.1).  With
 * private-key BFV the server cannot re-randomise c1 = sum_i a_i g_i on its
 * own, so the client also publishes a public key and the server adds a fresh
 * encryption of zero, (pk0 u + e1, pk1 u + e2), to every response block, e1
 * being the large flooding term.
 *
 * Public key from stream seed:
 *   a  uniform mod q_j, drawn directly in NTT form from (seed, A_PK, j), slot s
 *   e  centred binomial (eta = 21) from (seed, E_PK, 0), coefficient x
 *   pk1 = a,  pk0 = -a * s_hat + NTT(e)   (slot-wise), layout pk[c][j][s].
 */
void oracle_public_key(const oracle_params *P, const uint64_t *s_hat, uint64_t seed,
                       uint64_t *pk)
{
    uint32_t N = P->N, L = P->L;
    int64_t *ei = (int64_t *)malloc(sizeof(int64_t) * N);
    uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (uint32_t x = 0; x < N; x++) {
        uint64_t lo, hi;
        draw128(seed, PURPOSE_E_PK, 0, x, &lo, &hi);
        ei[x] = cbd21_of(lo);
    }
    for (uint32_t j = 0; j < L; j++) {
        uint64_t q = P->q[j];
        for (uint32_t x = 0; x < N; x++) e[x] = lift(ei[x], q);
        oracle_ntt(e, N, q, P->fwd + (size_t)j * N);
        uint64_t *p0 = pk + (size_t)j * N, *p1 = pk + ((size_t)L + j) * N;
        const uint64_t *sh = s_hat + (size_t)j * N;
        for (uint32_t s = 0; s < N; s++) {
            uint64_t lo, hi;
            draw128(seed, PURPOSE_A_PK, j, s, &lo, &hi);
            uint64_t a = uniform_of(lo, hi, q);
            p1[s] = a;
            p0[s] = add_mod(sub_mod(0, mul_mod(a, sh[s], q), q), e[s], q);
        }
    }
    free(e);
    free(ei);
}

/*
 * Re-randomisation (circuit privacy, Sec. 2.3) in the NTT domain, before the
 * inverse transform: for blocks k in [k0, k0 + nk) (global block index,
 * positions k N + x) of one query,
 *   u  ternary, (lo mod 3) - 1 of draw (seed, U, qid) at position k N + x,
 *   acc[k][c][j] += pk_c[j] * NTT(u)   (slot-wise), c = 0, 1.
 * acc is [nk][2][L][N], NTT form, modified in place.
 */
void oracle_rerandomize(const oracle_params *P, uint64_t *acc, const uint64_t *pk,
                        uint64_t seed, uint64_t qid, uint64_t k0, uint64_t nk)
{
    uint32_t N = P->N, L = P->L;
    int64_t *ui = (int64_t *)malloc(sizeof(int64_t) * N);
    uint64_t *u = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (uint64_t k = k0; k < k0 + nk; k++) {
        for (uint32_t x = 0; x < N; x++) {
            uint64_t lo, hi;
            draw128(seed, PURPOSE_U, qid, k * N + x, &lo, &hi);
            ui[x] = ternary_of(lo);
        }
        for (uint32_t j = 0; j < L; j++) {
            uint64_t q = P->q[j];
            for (uint32_t x = 0; x < N; x++) u[x] = lift(ui[x], q);
            oracle_ntt(u, N, q, P->fwd + (size_t)j * N);
            for (uint32_t c = 0; c < 2; c++) {
                uint64_t *a = acc + (((k - k0) * 2 + c) * L + j) * N;
                const uint64_t *p = pk + ((size_t)c * L + j) * N;
                for (uint32_t s = 0; s < N; s++) a[s] = add_mod(a[s], mul_mod(p[s], u[s], q), q);
            }
        }
    }
    free(u);
    free(ui);
}

/*
 * Flooding (circuit privacy by noise flooding, Sec. 2.3), in coefficient form
 * after the inverse transform and the mask:
 * at position k N + x of one query
 *   e1 = v - 2^F, v = the low F + 1 bits of the 256-bit integer
 *        lo_a + hi_a 2^64 + lo_b 2^128 + hi_b 2^192, (lo_a, hi_a) the draw
 *        (seed, FLOOD_LO, qid) and (lo_b, hi_b) the draw (seed, FLOOD_HI, qid)
 *        at that position: uniform in [-2^F, 2^F), F <= 255;
 *   e2 = centred binomial (eta = 21) of draw (seed, E2, qid);
 *   out[k][0][j][x] += e1 mod q_j,  out[k][1][j][x] += e2 mod q_j.
 */
void oracle_flood(const oracle_params *P, uint64_t *out, uint64_t seed, uint64_t qid,
                  uint64_t k0, uint64_t nk, uint32_t F)
{
    uint32_t N = P->N, L = P->L;
    for (uint64_t k = k0; k < k0 + nk; k++)
        for (uint32_t x = 0; x < N; x++) {
            uint64_t pos = k * N + x, w[4];
            draw128(seed, PURPOSE_FLOOD_LO, qid, pos, &w[0], &w[1]);
            draw128(seed, PURPOSE_FLOOD_HI, qid, pos, &w[2], &w[3]);
            /* keep bits 0 .. F of the 256-bit value */
            for (uint32_t b = 0; b < 4; b++) {
                int keep = (int)(F + 1) - 64 * (int)b;
                if (keep <= 0) w[b] = 0;
                else if (keep < 64) w[b] &= (1ull << keep) - 1;
            }
            uint64_t lo, hi;
            draw128(seed, PURPOSE_E2, qid, pos, &lo, &hi);
            int64_t e2 = cbd21_of(lo);
            for (uint32_t j = 0; j < L; j++) {
                uint64_t q = P->q[j];
                /* v mod q by Horner over the 64-bit words, then minus 2^F mod q */
                u128 r = 0;
                for (int b = 3; b >= 0; b--) r = ((r << 64) | w[b]) % q;
                u128 pf = 1;
                for (uint32_t i = 0; i < F; i++) pf = (pf * 2) % q;
                uint64_t e1 = sub_mod((uint64_t)r, (uint64_t)pf, q);
                size_t o0 = (((k - k0) * 2 + 0) * L + j) * N + x;
                size_t o1 = (((k - k0) * 2 + 1) * L + j) * N + x;
                out[o0] = add_mod(out[o0], e1, q);
                out[o1] = add_mod(out[o1], lift(e2, q), q);
            }
        }
}

/*
 * First half of decryption (Pi_ls step 4): v_j = c0 + c1 * s mod q_j in
 * coefficient form, for nk blocks of ct [k][2][L][N].  The product c1 * s is
 * the negacyclic product, taken through the NTT.  The CRT and the
 * scale-and-round step are done with exact big integers in oracle/bfv.py.
 */
void oracle_decrypt_phase(const oracle_params *P, const uint64_t *ct,
                          const int8_t *s, uint64_t nk, uint64_t *v)
{
    uint32_t N = P->N, L = P->L;
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint64_t *b = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (uint64_t k = 0; k < nk; k++)
        for (uint32_t j = 0; j < L; j++) {
            uint64_t q = P->q[j];
            const uint64_t *c0 = ct + ((k * 2 + 0) * L + j) * N;
            const uint64_t *c1 = ct + ((k * 2 + 1) * L + j) * N;
            for (uint32_t x = 0; x < N; x++) {
                a[x] = c1[x];
                b[x] = lift(s[x], q);
            }
            oracle_ntt(a, N, q, P->fwd + (size_t)j * N);
            oracle_ntt(b, N, q, P->fwd + (size_t)j * N);
            for (uint32_t x = 0; x < N; x++) a[x] = mul_mod(a[x], b[x], q);
            oracle_intt(a, N, q, P->inv + (size_t)j * N);
            uint64_t *o = v + (k * L + j) * N;
            for (uint32_t x = 0; x < N; x++) o[x] = add_mod(c0[x], a[x], q);
        }
    free(a);
    free(b);
}

/*
 * Schoolbook negacyclic product mod q: the definition of the product in
 * R_q = Z_q[x]/(x^N + 1) (Sec. 5.3), for the tests' cross-checks.
 */
void oracle_negacyclic_schoolbook(const uint64_t *a, const uint64_t *b,
                                  uint32_t N, uint64_t q, uint64_t *out)
{
    for (uint32_t x = 0; x < N; x++) out[x] = 0;
    for (uint32_t i = 0; i < N; i++)
        for (uint32_t j = 0; j < N; j++) {
            uint64_t p = mul_mod(a[i], b[j], q);
            uint32_t k = i + j;
            if (k < N) out[k] = add_mod(out[k], p, q);
            else out[k - N] = sub_mod(out[k - N], p, q);
        }
}
