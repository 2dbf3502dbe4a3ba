/*
 * fclsh_oracle.c -- plain, slow CPU oracle for Fast CoveringLSH (Pham & Pagh,
 * "Scalability and Total Recall with Fast CoveringLSH", arXiv 1602.02620).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything is written for clarity, not speed: one point, one table, one
 * coordinate at a time, 128-bit integers wherever a sum could grow, and no
 * blocking, fusion or reordering beyond what the paper's definitions state.
 *
 * Conventions (readings of the paper where it leaves a choice open):
 *   - A point is d bits packed LSB-first into ceil(d/64) uint64 words:
 *     coordinate i lives in word i/64, bit i%64.
 *   - Hadamard code entry C(v, j) = <a(j), v> mod 2 = parity(v & j), i.e. the
 *     Sylvester matrix in natural order (Sec. 2.4, Eq. 3; the printed C_{7,8}).
 *   - Table index tau = k*(W-1) + (v-1) for part k and code row v = 1..W-1.
 *
 * Parameters (perm, part_off, m, b) are inputs.  oracle_derive_params() draws
 * them from a seed with SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written
 * here from that paper's definition; the draw order is stated there.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* Parameters of one fcLSH index.  All arrays are owned by the caller. */
typedef struct {
    uint64_t P;              /* the prime of Eq. (1) */
    uint32_t d;              /* dimensionality of the input points */
    uint32_t t;              /* number of parts (Algorithm 1); 1 = no partitioning */
    uint32_t W;              /* code length 2^(r'+1) */
    uint32_t words;          /* uint64 words per packed point = ceil(d/64) */
    /* Positions: the D entries of the pre-processed vector (Algorithm 1).  D = d
       without replication (a permutation of the coordinates), D = d * rep with it
       (the vector written rep times in a row).  The arrays have D entries. */
    const uint32_t *perm;    /* [D]  position i of the pre-processed vector is coordinate perm[i] */
    const uint32_t *part_off;/* [t+1] part k = positions [part_off[k], part_off[k+1]) */
    const uint32_t *m;       /* [D]  m_k(i) in [0, W) for position i (column of the code) */
    const uint64_t *b;       /* [D]  b_k(i) in [0, P) for position i (Eq. 1; the seed vector of Algorithm 2) */
} oracle_params;

/* ---------------------------------------------------------------- SplitMix64 */
static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int bit_length(uint64_t x)
{
    int n = 0;
    while (x) { n++; x >>= 1; }
    return n;
}

/* Uniform integer in [0, P): take the top bit_length(P-1) bits, reject if >= P. */
static uint64_t draw_below_prime(uint64_t *state, uint64_t P)
{
    int bits = bit_length(P - 1);
    for (;;) {
        uint64_t u = sm64_next(state) >> (64 - bits);
        if (u < P) return u;
    }
}

/* Fisher-Yates shuffle of a[0..len): for i = len-1 down to 1, swap a[i] with a[next() % (i+1)]. */
static void fisher_yates(uint64_t *state, uint32_t *a, uint32_t len)
{
    for (uint32_t i = len; i-- > 1;) {
        uint32_t j = (uint32_t)(sm64_next(state) % (uint64_t)(i + 1));
        uint32_t tmp = a[i];
        a[i] = a[j];
        a[j] = tmp;
    }
}

/*
 * Draw pi, m_k and b_k from `seed` (Algorithm 1 pre-processing; Algorithm 2 choices of b and m).
 * Pre-processing (Algorithm 1): with rep > 1 (needs t = 1) the vector is replicated:
 * q^(rep) = q q ... q, so position i is coordinate i mod d, and nothing is drawn
 * (Example 3: 0011 replicated twice is 00110011).  Otherwise the positions are the
 * coordinates, permuted when t > 1.
 * Order of draws: (i) if t > 1, pi by Fisher-Yates over [d]; (ii) for each part k
 * in order: m_k, then b_k.  Part k < t-1 takes floor(D/t) consecutive positions
 * and the last part takes the remainder (Algorithm 1, partitioning).
 *   - d'_k <= W (specific construction, Algorithm 2): sigma = Fisher-Yates
 *     permutation of [W]; m_k(i) = sigma(i) for i < d'_k.
 *   - d'_k > W (general construction, Eq. 4): m_k(i) = 1 + next() % (W-1), i.e.
 *     uniform over the columns 1..W-1; column 0 is left out (Sec. 3.3, the sharper
 *     bound after Lemma 1).
 *   - b_k(i) uniform in [0, P) by rejection.
 * The arrays perm, m, b hold D = d * rep entries.  Returns 0 on success, -1 on bad arguments.
 */
int oracle_derive_params(uint64_t seed, uint32_t d, uint32_t t, uint32_t rep, uint32_t W, uint64_t P,
                         uint32_t *perm, uint32_t *part_off, uint32_t *m, uint64_t *b)
{
    if (d == 0 || t == 0 || t > d || rep == 0 || (rep > 1 && t > 1) || W < 2 || (W & (W - 1)) != 0 || P < 2)
        return -1;
    uint64_t state = seed;
    uint32_t D = d * rep;
    for (uint32_t copy = 0; copy < rep; copy++)          /* replication: copy after copy */
        for (uint32_t c = 0; c < d; c++) perm[copy * d + c] = c;
    if (t > 1) fisher_yates(&state, perm, d);
    uint32_t block = D / t;
    for (uint32_t k = 0; k < t; k++) part_off[k] = k * block;
    part_off[t] = D;
    uint32_t *sigma = (uint32_t *)malloc(sizeof(uint32_t) * W);
    if (!sigma) return -1;
    for (uint32_t k = 0; k < t; k++) {
        uint32_t lo = part_off[k], hi = part_off[k + 1], dk = hi - lo;
        if (dk <= W) {
            for (uint32_t j = 0; j < W; j++) sigma[j] = j;
            fisher_yates(&state, sigma, W);
            for (uint32_t i = 0; i < dk; i++) m[lo + i] = sigma[i];
        } else {
            for (uint32_t i = 0; i < dk; i++)
                m[lo + i] = 1 + (uint32_t)(sm64_next(&state) % (uint64_t)(W - 1));
        }
        for (uint32_t i = 0; i < dk; i++) b[lo + i] = draw_below_prime(&state, P);
    }
    free(sigma);
    return 0;
}

/* ---------------------------------------------------------------- helpers */
static int get_bit(const uint64_t *x, uint32_t i)
{
    return (int)((x[i >> 6] >> (i & 63)) & 1ULL);
}

static int parity32(uint32_t v)
{
    int p = 0;
    while (v) { p ^= 1; v &= v - 1; }
    return p;
}

/* Hadamard code entry: Had(v)_j = <a(j), v> mod 2 (Eq. 3), a(j) = binary form of j. */
static int had(uint32_t v, uint32_t j)
{
    return parity32(v & j);
}

static uint32_t num_tables(const oracle_params *p)
{
    return p->t * (p->W - 1);
}

/*
 * Direct route (bcLSH, the O(d L) way): build the covering hash vector g_v of
 * part k (Eq. 4: g_v,i = Had(v)_{m(i)}), AND it with the part's coordinates of x
 * (g_v(x) = g_v AND x, Sec. 2.3), then apply the universal hash of Eq. (1):
 * sum_i b_i * (g_v AND x)_i mod P.
 */
uint64_t oracle_key_direct(const oracle_params *p, const uint64_t *x, uint32_t tau)
{
    uint32_t L = p->W - 1;
    uint32_t k = tau / L;
    uint32_t v = tau % L + 1;
    u128 sum = 0;
    for (uint32_t i = p->part_off[k]; i < p->part_off[k + 1]; i++) {
        int g = had(v, p->m[i]);               /* g_v at position i of part k */
        int xi = get_bit(x, p->perm[i]);      /* coordinate of x at that position */
        int y = g & xi;                        /* (g_v AND x)_i */
        sum += (u128)p->b[i] * (u128)y;
    }
    return (uint64_t)(sum % p->P);
}

void oracle_keys_direct(const oracle_params *p, const uint64_t *pts, uint64_t n, uint64_t *keys)
{
    uint32_t T = num_tables(p);
    for (uint32_t tau = 0; tau < T; tau++)
        for (uint64_t i = 0; i < n; i++)
            keys[(uint64_t)tau * n + i] = oracle_key_direct(p, pts + i * p->words, tau);
}

/*
 * Fast Hadamard transform in place (unnormalised): after it, y_v = sum_j
 * (-1)^{<a(j), v>} t_j, i.e. y = H t with the Sylvester Hadamard matrix H.
 */
static void fht(i128 *t, uint32_t W)
{
    for (uint32_t h = 1; h < W; h <<= 1)
        for (uint32_t i = 0; i < W; i += 2 * h)
            for (uint32_t j = i; j < i + h; j++) {
                i128 a = t[j], c = t[j + h];
                t[j] = a + c;
                t[j + h] = a - c;
            }
}

/*
 * Algorithm 2 route for one point and one part k, in the algorithm's order:
 *   q~ = q * b (component-wise product);
 *   sketch t_j = sum_{i: m(i)=j} q~_i (general construction); for the specific
 *           construction column sigma(i) receives q~_i and the zero padding adds 0;
 *   h = 1/2 (||q~||_1 * 1 - FHT(t)) mod P;
 *   drop h_0, the entry of the all-zero code row.
 * No value is reduced before the final mod P; 128-bit integers keep every sum exact.
 * Writes the W-1 keys of part k to out[0..W-1).
 */
void oracle_keys_fht_part(const oracle_params *p, const uint64_t *x, uint32_t k, uint64_t *out)
{
    uint32_t W = p->W;
    i128 *t = (i128 *)calloc(W, sizeof(i128));
    i128 l1 = 0;
    for (uint32_t i = p->part_off[k]; i < p->part_off[k + 1]; i++) {
        i128 qt = (i128)p->b[i] * (i128)get_bit(x, p->perm[i]);   /* q~_i */
        l1 += qt;                                                  /* ||q~||_1 */
        t[p->m[i]] += qt;                                          /* sketch */
    }
    fht(t, W);
    for (uint32_t v = 1; v < W; v++) {
        i128 twice = l1 - t[v];         /* = 2 * sum_{j: C(v,j)=1} t_j, even and >= 0 */
        i128 half = twice / 2;
        out[v - 1] = (uint64_t)(half % (i128)p->P);
    }
    free(t);
}

void oracle_keys_fht(const oracle_params *p, const uint64_t *pts, uint64_t n, uint64_t *keys)
{
    uint32_t L = p->W - 1;
    uint64_t *row = (uint64_t *)malloc(sizeof(uint64_t) * L);
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t k = 0; k < p->t; k++) {
            oracle_keys_fht_part(p, pts + i * p->words, k, row);
            for (uint32_t v = 0; v < L; v++) keys[(uint64_t)(k * L + v) * n + i] = row[v];
        }
    free(row);
}

/* ---------------------------------------------------------------- tables */
typedef struct { uint64_t key; uint32_t id; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/*
 * One bucket table (Sec. 2.2: only non-empty buckets are stored): every point
 * id with its key in table tau, sorted by (key, id).  Equal keys form a bucket.
 */
void oracle_table(const oracle_params *p, const uint64_t *pts, uint64_t n, uint32_t tau,
                  uint64_t *keys_out, uint32_t *ids_out)
{
    kv_t *a = (kv_t *)malloc(sizeof(kv_t) * (n ? n : 1));
    for (uint64_t i = 0; i < n; i++) {
        a[i].key = oracle_key_direct(p, pts + i * p->words, tau);
        a[i].id = (uint32_t)i;
    }
    qsort(a, n, sizeof(kv_t), kv_cmp);
    for (uint64_t i = 0; i < n; i++) { keys_out[i] = a[i].key; ids_out[i] = a[i].id; }
    free(a);
}

static int hamming(const uint64_t *a, const uint64_t *b, uint32_t words)
{
    int dist = 0;
    for (uint32_t w = 0; w < words; w++) {
        uint64_t z = a[w] ^ b[w];
        while (z) { dist++; z &= z - 1; }
    }
    return dist;
}

/* First index in sorted keys[0..n) whose key is >= key. */
static uint64_t lower_bound_u64(const uint64_t *keys, uint64_t n, uint64_t key)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int u32_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Strategy 2 query (Sec. 2.2) with the cost steps of Sec. 4.1:
 *   S1: hash q into its key in every table (direct route);
 *   S2: look up the bucket of q in every probed table, merge with duplicate
 *       removal by an n-bit bitmap, counting #Collisions and #Candidates;
 *   S3: compute d(x, q) for each distinct candidate and report it if <= radius.
 * tab_keys/tab_ids are the T sorted tables from oracle_table(), each [n].
 * rows = 0 probes all W-1 tables of every part (the paper's query).  rows > 0
 * probes only the code rows v = 1..rows of every part: with rows =
 * 2^(floor(radius/t)+1) - 1 this is still exact, because a point within radius
 * of q is within floor(radius/t) of it on some part (pigeonhole, Sec. 3.1), and
 * Theorem 1 applied to the map m(i) mod 2^(floor(radius/t)+1) gives a row
 * v < 2^(floor(radius/t)+1) on which the two collide.  The counters then count
 * the probed tables only.
 * Results are sorted ascending.  Returns the number of results; writes up to
 * cap ids.  counters[0] = #Collisions, counters[1] = #Candidates.
 * tab_row (may be NULL): table tau is row tab_row[tau] of tab_keys/tab_ids, so that a
 * caller can pass only the probed tables; NULL means row tau.  A probed table without a
 * row (tab_row[tau] = 0xFFFFFFFF) makes the query fail: it returns UINT64_MAX.
 */
static uint64_t query_core(const oracle_params *p, const uint64_t *pts, uint64_t n,
                           const uint64_t *tab_keys, const uint32_t *tab_ids, const uint32_t *tab_row,
                           const uint64_t *q, uint32_t radius, uint32_t rows,
                           uint32_t *out, uint64_t cap, uint64_t *counters)
{
    uint32_t T = num_tables(p);
    uint64_t *qkeys = (uint64_t *)malloc(sizeof(uint64_t) * T);
    unsigned char *bitmap = (unsigned char *)calloc((n + 7) / 8 + 1, 1);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint64_t ncand = 0, ncoll = 0, nres = 0;

    for (uint32_t tau = 0; tau < T; tau++)                        /* S1 */
        qkeys[tau] = oracle_key_direct(p, q, tau);

    for (uint32_t tau = 0; tau < T; tau++) {                      /* S2 */
        uint32_t v = tau % (p->W - 1) + 1;                        /* code row of table tau */
        if (rows && v > rows) continue;
        uint64_t row = tab_row ? tab_row[tau] : tau;
        if (row == 0xFFFFFFFFu) { ncoll = UINT64_MAX; break; }   /* a probed table was not given */
        const uint64_t *keys = tab_keys + row * n;
        const uint32_t *ids = tab_ids + row * n;
        for (uint64_t e = lower_bound_u64(keys, n, qkeys[tau]); e < n && keys[e] == qkeys[tau]; e++) {
            uint32_t id = ids[e];
            ncoll++;
            if (!(bitmap[id >> 3] & (1u << (id & 7)))) {
                bitmap[id >> 3] |= (unsigned char)(1u << (id & 7));
                cand[ncand++] = id;
            }
        }
    }

    if (ncoll == UINT64_MAX) {
        free(qkeys);
        free(bitmap);
        free(cand);
        return UINT64_MAX;
    }
    for (uint64_t c = 0; c < ncand; c++) {                        /* S3 */
        uint32_t id = cand[c];
        if (hamming(q, pts + (uint64_t)id * p->words, p->words) <= (int)radius) {
            if (nres < cap) out[nres] = id;
            nres++;
        }
    }
    if (nres <= cap) qsort(out, nres, sizeof(uint32_t), u32_cmp);
    counters[0] = ncoll;
    counters[1] = ncand;
    free(qkeys);
    free(bitmap);
    free(cand);
    return nres;
}

uint64_t oracle_query_rows(const oracle_params *p, const uint64_t *pts, uint64_t n,
                           const uint64_t *tab_keys, const uint32_t *tab_ids,
                           const uint64_t *q, uint32_t radius, uint32_t rows,
                           uint32_t *out, uint64_t cap, uint64_t *counters)
{
    return query_core(p, pts, n, tab_keys, tab_ids, NULL, q, radius, rows, out, cap, counters);
}

/* The same query with only some tables given (tab_row as in query_core). */
uint64_t oracle_query_listed(const oracle_params *p, const uint64_t *pts, uint64_t n,
                             const uint64_t *tab_keys, const uint32_t *tab_ids, const uint32_t *tab_row,
                             const uint64_t *q, uint32_t radius, uint32_t rows,
                             uint32_t *out, uint64_t cap, uint64_t *counters)
{
    return query_core(p, pts, n, tab_keys, tab_ids, tab_row, q, radius, rows, out, cap, counters);
}

uint64_t oracle_query(const oracle_params *p, const uint64_t *pts, uint64_t n,
                      const uint64_t *tab_keys, const uint32_t *tab_ids,
                      const uint64_t *q, uint32_t radius,
                      uint32_t *out, uint64_t cap, uint64_t *counters)
{
    return oracle_query_rows(p, pts, n, tab_keys, tab_ids, q, radius, 0, out, cap, counters);
}

/*
 * The plain definition of the answer (Definition 2 with delta = 0; the ground
 * truth of Sec. 4.2 is computed the same way): every id whose Hamming distance
 * to q is at most radius, ascending.  Returns the count; writes up to cap ids.
 */
uint64_t oracle_linear_scan(const uint64_t *pts, uint64_t n, uint32_t words,
                            const uint64_t *q, uint32_t radius, uint32_t *out, uint64_t cap)
{
    uint64_t nres = 0;
    for (uint64_t i = 0; i < n; i++)
        if (hamming(q, pts + i * words, words) <= (int)radius) {
            if (nres < cap) out[nres] = (uint32_t)i;
            nres++;
        }
    return nres;
}

/* Hamming distance of two packed vectors (exposed for tests). */
int oracle_hamming(const uint64_t *a, const uint64_t *b, uint32_t words)
{
    return hamming(a, b, words);
}

/* The first n outputs of SplitMix64 started at `seed` (exposed for tests). */
void oracle_splitmix64(uint64_t seed, uint64_t n, uint64_t *out)
{
    uint64_t state = seed;
    for (uint64_t i = 0; i < n; i++) out[i] = sm64_next(&state);
}
