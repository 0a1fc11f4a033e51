/*
 * Plain CPU oracle for the level-wise wavelet tree of "GPU Implementation of
 * the Wavelet Tree" (arXiv 2505.03372).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * library; the two only ever see the same seeded inputs.
 *
 * Two independent oracles live here:
 *
 *  O1 (definitional, Section 1): access(i) = S[i]; rank_c(i) = #{j < i :
 *     S[j] = c} for 0 <= i <= n; select_c(j) = position of the j-th (1-based)
 *     occurrence of c.  Built from occurrence lists (a counting sort of the
 *     positions by symbol); rank is a lower bound in the list, select an index.
 *
 *  O2 (the method, Sections 4 and 5): a naive level-wise wavelet tree with
 *     reduced codes.  Codes come from the recursive alphabet split of Section
 *     5.1 (a node [a,b) sends [a, a+prevPow2(b-a)) left, the rest right).
 *     Level l's bit array is bit l (from the top) of the code of every symbol
 *     of S stably sorted by its first l code bits (Algorithm 4), recomputed
 *     from S at every level by a counting sort.  Binary rank/select run on a
 *     plain cumulative popcount per 64-bit word, not on the L1/L2 blocks.  The
 *     L1/L2 counters, the select samples and the node-start ranks are produced
 *     by direct counting, only to be compared with the GPU's.  Queries follow
 *     Algorithms 5, 6, 7 and 8 read this way: the access loop runs over
 *     l in [0, L), its "index" update means i, and a node of two symbols is
 *     decided by one bit (no bit is read at a node of one symbol); the rank
 *     walk stops at a node of one symbol (width <= 1, not <= 0); getNodeStart
 *     encodes the start symbol passed in and "rightmost" means the first l code
 *     bits are all ones; a level's bit is bit L-1-l of the left-aligned code.
 *
 * Parity status: every function here is pinned by tests/test_oracle_pins.py
 * (brute force on tiny inputs, the worked example of Section 5, closed forms
 * and invariants); none is "parity unpinned".
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_L1_BITS 65536u /* Section 4.1: L1-block size */
#define ORC_L2_BITS 512u   /* Section 6.2/6.3: |L2| = 512 in every experiment */

/* ------------------------------------------------------------------------- */
/* small helpers                                                              */
/* ------------------------------------------------------------------------- */

static uint64_t sym_at(const void* S, int w, uint64_t j) {
    if (w == 1) return ((const uint8_t*)S)[j];
    if (w == 2) return ((const uint16_t*)S)[j];
    return ((const uint32_t*)S)[j];
}

static int is_pow2(uint64_t x) { return x != 0 && (x & (x - 1)) == 0; }

/* Largest power of two strictly below x, for x >= 2 (prevPowTwo, Section 5). */
static uint64_t prev_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p * 2 < x) p *= 2;
    return p;
}

/* ceil(lg x) for x >= 1 */
static uint32_t ceil_lg(uint64_t x) {
    uint32_t l = 0;
    while (((uint64_t)1 << l) < x) l++;
    return l;
}

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

/* ------------------------------------------------------------------------- */
/* threads: the O2 build, its sample export and the query loops split their   */
/* index ranges over host threads; results do not depend on the thread count  */
/* ------------------------------------------------------------------------- */

#define ORC_MAX_THREADS 256

/* Threads to use: requested > 0, else the online CPUs; 1 for small work. */
static int orc_threads(int requested, uint64_t work) {
    long nt = requested > 0 ? requested : sysconf(_SC_NPROCESSORS_ONLN);
    if (requested <= 0 && work < ((uint64_t)1 << 16)) nt = 1;
    if (nt < 1) nt = 1;
    if (nt > ORC_MAX_THREADS) nt = ORC_MAX_THREADS;
    return (int)nt;
}

/* Run fn on jobs[0..nt) (each job_size bytes), job 0 on the calling thread.
 * A job whose thread cannot be started runs on the calling thread too.     */
static void orc_run(void* (*fn)(void*), void* jobs, size_t job_size, int nt) {
    pthread_t th[ORC_MAX_THREADS];
    int ok[ORC_MAX_THREADS];
    for (int i = 1; i < nt; i++) ok[i] = pthread_create(&th[i], NULL, fn, (char*)jobs + (size_t)i * job_size) == 0;
    fn(jobs);
    for (int i = 1; i < nt; i++) {
        if (ok[i]) pthread_join(th[i], NULL);
        else fn((char*)jobs + (size_t)i * job_size);
    }
}

/* [lo, hi) of part i of nt equal parts of [0, n) */
static void orc_split(uint64_t n, int nt, int i, uint64_t* lo, uint64_t* hi) {
    *lo = n / (uint64_t)nt * (uint64_t)i + (n % (uint64_t)nt < (uint64_t)i ? n % (uint64_t)nt : (uint64_t)i);
    *hi = *lo + n / (uint64_t)nt + ((uint64_t)i < n % (uint64_t)nt ? 1 : 0);
}

/* ------------------------------------------------------------------------- */
/* Codes                                                                      */
/* ------------------------------------------------------------------------- */

/* Recursive split of Section 5.1: node [a,b) with b-a >= 2 sends
 * [a, a+prevPow2(b-a)) to the left child (bit 0) and the rest right (bit 1).
 * A symbol's code is its root-to-leaf path, its length the leaf depth.       */
static void split_rec(uint64_t a, uint64_t b, uint32_t depth, uint64_t path,
                      uint64_t* code, uint8_t* len) {
    if (b - a == 1) {
        code[a] = path;
        len[a] = (uint8_t)depth;
        return;
    }
    uint64_t p = prev_pow2(b - a);
    split_rec(a, a + p, depth + 1, path << 1, code, len);
    split_rec(a + p, b, depth + 1, (path << 1) | 1u, code, len);
}

/* Codes left-aligned in L = ceil(lg sigma) bits; returns L. */
int orc_codes_split(uint32_t sigma, uint64_t* code, uint8_t* len, uint32_t* L_out) {
    if (sigma == 0) return -1;
    uint32_t L = ceil_lg(sigma);
    *L_out = L;
    if (sigma == 1) {
        code[0] = 0;
        len[0] = 0;
        return 0;
    }
    split_rec(0, sigma, 0, 0, code, len);
    for (uint32_t s = 0; s < sigma; s++) code[s] <<= (L - len[s]);
    return 0;
}

/* Algorithm 3 (createCodes), step by step, with these readings of the
 * garbled listing: codes are indexed by symbol; every symbol starts with its
 * own value as code and L as length (the identity code that symbols below
 * prevPow2(sigma) keep); the "~" is a bitwise NOT, so the term keeps the
 * first start_bit bits of the symbol's current code.                         */
int orc_codes_alg3(uint32_t sigma, uint64_t* code, uint8_t* len, uint32_t* L_out) {
    if (sigma == 0) return -1;
    uint32_t total_num_bits = ceil_lg(sigma);
    *L_out = total_num_bits;
    for (uint32_t s = 0; s < sigma; s++) {
        code[s] = s;
        len[s] = (uint8_t)total_num_bits;
    }
    if (sigma == 1 || is_pow2(sigma)) return 0;
    uint32_t alphabet_start_bit = total_num_bits - 1;
    uint32_t start_bit = 0;
    uint64_t start_i = 0;
    uint32_t code_len = total_num_bits;
    uint64_t num_codes = sigma;
    do {
        for (int i = (int)code_len - 1; i >= 1; i--) {
            uint64_t pow_two = (uint64_t)1 << i;
            if (num_codes <= pow_two) break;
            num_codes -= pow_two;
            start_i += pow_two;
            start_bit += 1;
        }
        if (num_codes == 1) {
            code_len = 1;
            len[sigma - 1] = (uint8_t)start_bit;
            code[sigma - 1] = (((uint64_t)1 << start_bit) - 1) << (alphabet_start_bit + 1 - start_bit);
        } else {
            code_len = ceil_lg(num_codes);
            for (uint64_t i = sigma - num_codes; i < sigma; i++) {
                uint64_t local_code = i - start_i;
                local_code <<= (total_num_bits - start_bit - code_len);
                local_code += (~((((uint64_t)1) << (total_num_bits - start_bit)) - 1)) & code[i];
                code[i] = local_code;
                len[i] = (uint8_t)(start_bit + code_len);
            }
        }
    } while (code_len != 1);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O1: occurrence lists                                                       */
/* ------------------------------------------------------------------------- */

/* C[c] = #{j : S[j] < c} for c in [0, sigma]; occ[C[c] + k] = position of the
 * (k+1)-th occurrence of c.  Returns -1 if some S[j] >= sigma.              */
int orc_o1_build(const void* S, int w, uint64_t n, uint32_t sigma, uint64_t* C, uint64_t* occ) {
    uint64_t* cur = (uint64_t*)calloc((size_t)sigma + 1, sizeof(uint64_t));
    if (!cur) return -2;
    memset(C, 0, ((size_t)sigma + 1) * sizeof(uint64_t));
    for (uint64_t j = 0; j < n; j++) {
        uint64_t s = sym_at(S, w, j);
        if (s >= sigma) {
            free(cur);
            return -1;
        }
        C[s + 1]++;
    }
    for (uint32_t c = 0; c < sigma; c++) C[c + 1] += C[c];
    for (uint32_t c = 0; c <= sigma; c++) cur[c] = C[c];
    for (uint64_t j = 0; j < n; j++) occ[cur[sym_at(S, w, j)]++] = j;
    free(cur);
    return 0;
}

void orc_o1_access(const void* S, int w, uint64_t n, const uint64_t* idx, uint64_t q, uint32_t* out) {
    for (uint64_t k = 0; k < q; k++) out[k] = idx[k] < n ? (uint32_t)sym_at(S, w, idx[k]) : UINT32_MAX;
}

void orc_o1_rank(const uint64_t* C, const uint64_t* occ, uint64_t n, uint32_t sigma,
                 const uint32_t* c, const uint64_t* i, uint64_t q, uint64_t* out) {
    for (uint64_t k = 0; k < q; k++) {
        if (c[k] >= sigma || i[k] > n) {
            out[k] = UINT64_MAX;
            continue;
        }
        /* number of occurrences of c[k] at positions < i[k] */
        uint64_t lo = C[c[k]], hi = C[c[k] + 1];
        uint64_t a = lo, b = hi;
        while (a < b) {
            uint64_t m = a + (b - a) / 2;
            if (occ[m] < i[k]) a = m + 1;
            else b = m;
        }
        out[k] = a - lo;
    }
}

void orc_o1_select(const uint64_t* C, const uint64_t* occ, uint32_t sigma,
                   const uint32_t* c, const uint64_t* j, uint64_t q, uint64_t* out) {
    for (uint64_t k = 0; k < q; k++) {
        if (c[k] >= sigma || j[k] == 0 || j[k] > C[c[k] + 1] - C[c[k]]) {
            out[k] = UINT64_MAX;
            continue;
        }
        out[k] = occ[C[c[k]] + j[k] - 1];
    }
}

/* ------------------------------------------------------------------------- */
/* O2: naive level-wise wavelet tree                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint64_t size;   /* bits in this level: #{j : len(S[j]) > l} */
    uint64_t nwords; /* ceil(size / 64) */
    uint64_t* bits;  /* LSB-first, tail bits zero */
    uint64_t* pc;    /* pc[w] = ones in words [0, w), nwords + 1 entries */
    uint64_t ones;
} orc_level;

typedef struct orc_tree {
    uint64_t n;
    uint32_t sigma, L, K;
    uint64_t* code; /* left-aligned in L bits */
    uint8_t* len;
    uint64_t* C; /* sigma + 1 */
    orc_level* lv;
} orc_tree;

static int bit_at(const orc_level* v, uint64_t i) { return (int)((v->bits[i >> 6] >> (i & 63)) & 1u); }

/* Binary rank_1 over the plain cumulative popcount (Section 4 definition:
 * ones in B[0, i), 0 <= i <= size).                                          */
static uint64_t lv_rank1(const orc_level* v, uint64_t i) {
    uint64_t w = i >> 6, r = i & 63;
    uint64_t res = v->pc[w];
    if (r) res += (uint64_t)popc64(v->bits[w] & ((((uint64_t)1) << r) - 1));
    return res;
}
static uint64_t lv_rank(const orc_level* v, int b, uint64_t i) { return b ? lv_rank1(v, i) : i - lv_rank1(v, i); }

/* Binary select: position of the k-th (1-based) bit equal to b; k must be in
 * [1, count_b].  Binary search over the per-word counts, then a bit scan.   */
static uint64_t lv_select(const orc_level* v, int b, uint64_t k) {
    uint64_t lo = 0, hi = v->nwords; /* find last word w with count_b(words < w) < k */
    while (hi - lo > 1) {
        uint64_t m = lo + (hi - lo) / 2;
        uint64_t cb = b ? v->pc[m] : 64 * m - v->pc[m];
        if (cb < k) lo = m;
        else hi = m;
    }
    uint64_t before = b ? v->pc[lo] : 64 * lo - v->pc[lo];
    uint64_t p = lo * 64;
    for (;; p++) {
        if (bit_at(v, p) == b) {
            before++;
            if (before == k) return p;
        }
    }
}

/* One thread's share of a level: positions [a, b) of S (count and scatter)
 * and words [w0, w1) of the level (packing).                                 */
typedef struct {
    const orc_tree* t;
    const void* S;
    int w;
    uint32_t l;
    uint64_t a, b;
    uint64_t* cnt;  /* bucket counts of this share, then its first slot per bucket */
    uint64_t size;  /* symbols of the share whose code is longer than l */
    uint8_t* tmp;   /* one byte per position of the level: its bit */
    orc_level* v;
    uint64_t w0, w1;
} orc_lvl_job;

static void* orc_lvl_count(void* p) {
    orc_lvl_job* j = (orc_lvl_job*)p;
    const orc_tree* t = j->t;
    for (uint64_t i = j->a; i < j->b; i++) {
        uint64_t s = sym_at(j->S, j->w, i);
        j->cnt[t->code[s] >> (t->L - j->l)]++;
        if (t->len[s] > j->l) j->size++;
    }
    return NULL;
}

static void* orc_lvl_scatter(void* p) {
    orc_lvl_job* j = (orc_lvl_job*)p;
    const orc_tree* t = j->t;
    const uint64_t size = j->v->size;
    for (uint64_t i = j->a; i < j->b; i++) {
        uint64_t s = sym_at(j->S, j->w, i);
        uint64_t pos = j->cnt[t->code[s] >> (t->L - j->l)]++;
        if (t->len[s] > j->l && pos < size) j->tmp[pos] = (uint8_t)((t->code[s] >> (t->L - 1 - j->l)) & 1u);
    }
    return NULL;
}

static void* orc_lvl_pack(void* p) {
    orc_lvl_job* j = (orc_lvl_job*)p;
    const uint64_t size = j->v->size;
    for (uint64_t k = j->w0; k < j->w1; k++) {
        uint64_t x = 0;
        for (uint64_t b = 0; b < 64 && k * 64 + b < size; b++)
            if (j->tmp[k * 64 + b]) x |= ((uint64_t)1) << b;
        j->v->bits[k] = x;
    }
    return NULL;
}

orc_tree* orc_o2_build_mt(const void* S, int w, uint64_t n, uint32_t sigma, uint32_t K, int threads) {
    if (sigma == 0 || K == 0) return NULL;
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->sigma = sigma;
    t->K = K;
    t->code = (uint64_t*)malloc(sizeof(uint64_t) * sigma);
    t->len = (uint8_t*)malloc(sigma);
    orc_codes_split(sigma, t->code, t->len, &t->L);
    t->C = (uint64_t*)calloc((size_t)sigma + 1, sizeof(uint64_t));
    for (uint64_t j = 0; j < n; j++) {
        uint64_t s = sym_at(S, w, j);
        if (s >= sigma) {
            free(t->code);
            free(t->len);
            free(t->C);
            free(t);
            return NULL;
        }
        t->C[s + 1]++;
    }
    for (uint32_t c = 0; c < sigma; c++) t->C[c + 1] += t->C[c];
    uint32_t L = t->L;
    t->lv = (orc_level*)calloc(L ? L : 1, sizeof(orc_level));
    const int nt_all = orc_threads(threads, n);
    uint8_t* tmp = (uint8_t*)malloc(n ? n : 1);
    orc_lvl_job jobs[ORC_MAX_THREADS];
    for (uint32_t l = 0; l < L; l++) {
        orc_level* v = &t->lv[l];
        /* stable counting sort of S by the first l code bits (Algorithm 4);
         * finished codes sort behind all unfinished ones because code lengths
         * never increase with the symbol.  Each thread counts its range of
         * positions per bucket; slots are handed out bucket by bucket and,
         * within a bucket, range by range, which keeps the order stable.     */
        uint64_t nb = (uint64_t)1 << l;
        int nt = nt_all;
        while (nt > 1 && nb * (uint64_t)nt > ((uint64_t)1 << 26)) nt--;  /* bounded count arrays */
        uint64_t* cnt = (uint64_t*)calloc(nb * (uint64_t)nt, sizeof(uint64_t));
        for (int i = 0; i < nt; i++) {
            memset(&jobs[i], 0, sizeof(jobs[i]));
            jobs[i].t = t;
            jobs[i].S = S;
            jobs[i].w = w;
            jobs[i].l = l;
            jobs[i].cnt = cnt + nb * (uint64_t)i;
            jobs[i].tmp = tmp;
            jobs[i].v = v;
            orc_split(n, nt, i, &jobs[i].a, &jobs[i].b);
        }
        orc_run(orc_lvl_count, jobs, sizeof(jobs[0]), nt);
        uint64_t size = 0, run = 0;
        for (int i = 0; i < nt; i++) size += jobs[i].size;
        for (uint64_t k = 0; k < nb; k++)
            for (int i = 0; i < nt; i++) {
                uint64_t c = jobs[i].cnt[k];
                jobs[i].cnt[k] = run;
                run += c;
            }
        v->size = size;
        v->nwords = (size + 63) / 64;
        v->bits = (uint64_t*)calloc(v->nwords + 1, sizeof(uint64_t));
        orc_run(orc_lvl_scatter, jobs, sizeof(jobs[0]), nt);
        for (int i = 0; i < nt; i++) orc_split(v->nwords, nt, i, &jobs[i].w0, &jobs[i].w1);
        orc_run(orc_lvl_pack, jobs, sizeof(jobs[0]), nt);
        free(cnt);
        v->pc = (uint64_t*)malloc(sizeof(uint64_t) * (v->nwords + 2));
        v->pc[0] = 0;
        for (uint64_t k = 0; k <= v->nwords; k++) v->pc[k + 1] = v->pc[k] + (uint64_t)popc64(v->bits[k]);
        v->ones = v->pc[v->nwords];
    }
    free(tmp);
    return t;
}

orc_tree* orc_o2_build(const void* S, int w, uint64_t n, uint32_t sigma, uint32_t K) {
    return orc_o2_build_mt(S, w, n, sigma, K, 0);
}

void orc_o2_free(orc_tree* t) {
    if (!t) return;
    for (uint32_t l = 0; l < t->L; l++) {
        free(t->lv[l].bits);
        free(t->lv[l].pc);
    }
    free(t->lv);
    free(t->code);
    free(t->len);
    free(t->C);
    free(t);
}

uint32_t orc_o2_levels(const orc_tree* t) { return t->L; }
uint64_t orc_o2_level_size(const orc_tree* t, uint32_t l) { return l < t->L ? t->lv[l].size : 0; }
uint64_t orc_o2_level_ones(const orc_tree* t, uint32_t l) { return l < t->L ? t->lv[l].ones : 0; }

uint64_t orc_o2_rank_b(const orc_tree* t, uint32_t l, uint32_t b, uint64_t i) {
    if (l >= t->L || i > t->lv[l].size) return UINT64_MAX;
    return lv_rank(&t->lv[l], (int)b, i);
}
uint64_t orc_o2_select_b(const orc_tree* t, uint32_t l, uint32_t b, uint64_t k) {
    if (l >= t->L) return UINT64_MAX;
    const orc_level* v = &t->lv[l];
    uint64_t tot = b ? v->ones : v->size - v->ones;
    if (k == 0 || k > tot) return UINT64_MAX;
    return lv_select(v, (int)b, k);
}

/* Node table by recursion over the alphabet split: for every internal node
 * [a,b) at depth d with path p (d bits): start = C[a] (first position of the
 * node in level d), r0 = rank_0(d, C[a]), mid = C[a + prevPow2(b - a)].     */
static void nodes_rec(const orc_tree* t, uint64_t a, uint64_t b, uint32_t d, uint64_t p, uint64_t* out) {
    if (b - a < 2) return;
    uint64_t* e = out + 4 * ((((uint64_t)1) << d) - 1 + p);
    e[0] = t->C[a];
    e[1] = lv_rank(&t->lv[d], 0, t->C[a]);
    e[2] = t->C[a + prev_pow2(b - a)];
    e[3] = 1;
    uint64_t m = a + prev_pow2(b - a);
    nodes_rec(t, a, m, d + 1, p << 1, out);
    nodes_rec(t, m, b, d + 1, (p << 1) | 1u, out);
}

/* One thread's range of a level for the sample export. */
typedef struct {
    const orc_level* v;
    int b;
    uint64_t K, p0, p1, before, cnt;
    uint64_t* out;
} orc_smp_job;

static void* orc_smp_scan(void* p) {
    orc_smp_job* j = (orc_smp_job*)p;
    uint64_t seen = j->before;
    for (uint64_t q = j->p0; q < j->p1; q++) {
        if (bit_at(j->v, q) == j->b) {
            seen++;
            if (seen % j->K == 0 && seen / j->K < j->cnt) j->out[seen / j->K] = q;
        }
    }
    return NULL;
}

/* Logical contents for comparison with the GPU export.
 * what: 0 level bits (u64 words, ceil(size/64))
 *       1 L1 counters (u64, floor(size/65536) + 1): ones in B[0, 65536 k)
 *       2 L2 counters (u16, floor(size/512) + 1): ones from the start of the
 *         enclosing L1 block to 512 m
 *       3 zero samples (u64, floor(zeros/K) + 1): [0] = 0, [m] = position of
 *         the (m K)-th zero
 *       4 one samples (u64, floor(ones/K) + 1), likewise for ones
 *       5 C (u64, sigma + 1)      6 codes (u64, sigma)   7 lengths (u8, sigma)
 *       8 node table (u64 x 4 per slot, 2^L - 1 slots in heap order
 *         (level d, path p) -> 2^d - 1 + p): start, r0, mid, valid
 * Returns the element count; dst may be NULL to query it.                   */
uint64_t orc_o2_export(const orc_tree* t, uint32_t l, uint32_t what, void* dst) {
    if (what == 5) {
        if (dst) memcpy(dst, t->C, sizeof(uint64_t) * ((size_t)t->sigma + 1));
        return (uint64_t)t->sigma + 1;
    }
    if (what == 6) {
        if (dst) memcpy(dst, t->code, sizeof(uint64_t) * t->sigma);
        return t->sigma;
    }
    if (what == 7) {
        if (dst) memcpy(dst, t->len, t->sigma);
        return t->sigma;
    }
    if (what == 8) {
        uint64_t slots = t->L ? ((((uint64_t)1) << t->L) - 1) : 0;
        if (dst && slots) {
            memset(dst, 0, sizeof(uint64_t) * 4 * slots);
            nodes_rec(t, 0, t->sigma, 0, 0, (uint64_t*)dst);
        }
        return slots;
    }
    if (l >= t->L) return 0;
    const orc_level* v = &t->lv[l];
    if (what == 0) {
        if (dst) memcpy(dst, v->bits, sizeof(uint64_t) * v->nwords);
        return v->nwords;
    }
    if (what == 1) {
        uint64_t cnt = v->size / ORC_L1_BITS + 1;
        if (dst) {
            uint64_t* o = (uint64_t*)dst;
            for (uint64_t k = 0; k < cnt; k++) o[k] = lv_rank1(v, k * ORC_L1_BITS);
        }
        return cnt;
    }
    if (what == 2) {
        uint64_t cnt = v->size / ORC_L2_BITS + 1;
        if (dst) {
            uint16_t* o = (uint16_t*)dst;
            for (uint64_t m = 0; m < cnt; m++) {
                uint64_t pos = m * ORC_L2_BITS;
                uint64_t blk = (pos / ORC_L1_BITS) * ORC_L1_BITS;
                o[m] = (uint16_t)(lv_rank1(v, pos) - lv_rank1(v, blk));
            }
        }
        return cnt;
    }
    if (what == 3 || what == 4) {
        int b = what == 4;
        uint64_t tot = b ? v->ones : v->size - v->ones;
        uint64_t cnt = tot / t->K + 1;
        if (dst) {
            uint64_t* o = (uint64_t*)dst;
            o[0] = 0;
            /* direct count: walk every bit once, each thread over its own
             * range of positions after counting the b-bits before it        */
            orc_smp_job jobs[ORC_MAX_THREADS];
            const int nt = orc_threads(0, v->size);
            for (int i = 0; i < nt; i++) {
                uint64_t w0, w1;
                orc_split(v->nwords, nt, i, &w0, &w1);
                jobs[i].v = v;
                jobs[i].b = b;
                jobs[i].K = t->K;
                jobs[i].p0 = w0 * 64;
                jobs[i].p1 = w1 * 64 < v->size ? w1 * 64 : v->size;
                jobs[i].before = 0;
                jobs[i].out = o;
                jobs[i].cnt = cnt;
            }
            uint64_t run = 0;
            for (int i = 0; i < nt; i++) {
                jobs[i].before = run;
                uint64_t ones = v->pc[jobs[i].p1 / 64] - v->pc[jobs[i].p0 / 64];
                if (jobs[i].p1 % 64) ones += (uint64_t)popc64(v->bits[jobs[i].p1 / 64] & ((((uint64_t)1) << (jobs[i].p1 % 64)) - 1));
                run += b ? ones : (jobs[i].p1 - jobs[i].p0) - ones;
            }
            orc_run(orc_smp_scan, jobs, sizeof(jobs[0]), nt);
        }
        return cnt;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* O2 queries: Algorithms 5-8                                                 */
/* ------------------------------------------------------------------------- */

/* Algorithm 5 (access).  Loop over l in [0, L); at a node of at most two
 * symbols one bit decides; the update of the in-node index uses i (the
 * listing's "index" is i).                                                   */
static uint32_t o2_access1(const orc_tree* t, uint64_t i) {
    uint64_t start_symbol = 0, end_symbol = t->sigma;
    for (uint32_t l = 0; l < t->L; l++) {
        uint64_t counts = t->C[start_symbol];
        if (end_symbol - start_symbol <= 2) {
            if (end_symbol - start_symbol > 1 && bit_at(&t->lv[l], counts + i) == 1) return (uint32_t)(start_symbol + 1);
            return (uint32_t)start_symbol;
        }
        uint64_t start = lv_rank(&t->lv[l], 0, counts);
        uint64_t pos = lv_rank(&t->lv[l], 0, counts + i);
        uint64_t diff = prev_pow2(end_symbol - start_symbol);
        if (bit_at(&t->lv[l], counts + i) == 0) {
            i = pos - start;
            end_symbol = start_symbol + diff;
        } else {
            i = i - (pos - start);
            start_symbol = start_symbol + diff;
        }
    }
    return (uint32_t)start_symbol; /* sigma == 1: the only symbol */
}

/* Algorithm 6 (rank).  The walk stops once the node holds a single symbol
 * (a leaf), which for reduced codes can happen before level L.               */
static uint64_t o2_rank1(const orc_tree* t, uint64_t c, uint64_t i) {
    uint64_t start_symbol = 0, end_symbol = t->sigma, result = i;
    for (uint32_t l = 0; l < t->L; l++) {
        if (end_symbol - start_symbol <= 1) break;
        uint64_t counts = t->C[start_symbol];
        uint64_t start = lv_rank(&t->lv[l], 0, counts);
        uint64_t pos = lv_rank(&t->lv[l], 0, counts + result);
        uint64_t split_symbol = start_symbol + prev_pow2(end_symbol - start_symbol);
        if (c < split_symbol) {
            result = pos - start;
            end_symbol = split_symbol;
        } else {
            result = result - (pos - start);
            start_symbol = split_symbol;
        }
    }
    return result;
}

/* Algorithm 8 (getNodeStart): first symbol of the level-l node that holds the
 * node starting at symbol c.  encode() is applied to c, the start symbol that
 * is passed in; "rightmost" means the first l code bits are all ones.        */
static uint64_t o2_node_start(const orc_tree* t, uint64_t c, uint32_t l) {
    uint64_t node_start = 0;
    if (is_pow2(t->sigma)) {
        uint64_t node_len_at_level = ((uint64_t)1) << (t->L - l);
        node_start = c & ~(node_len_at_level - 1);
    } else {
        uint64_t code = t->code[c];
        uint32_t len = t->len[c];
        int is_rightmost = popc64(code >> (t->L - l)) == (int)l;
        if (is_rightmost) {
            for (uint32_t k = 0; k < l; k++) node_start += prev_pow2(t->sigma - node_start);
        } else {
            node_start = c - (((uint64_t)1) << (len - l - 1));
        }
    }
    return node_start;
}

uint64_t orc_o2_node_start(const orc_tree* t, uint64_t c, uint32_t l) { return o2_node_start(t, c, l); }

/* Algorithm 7 (select), leaf to root over levels len(c)-1 .. 0. */
static uint64_t o2_select1(const orc_tree* t, uint64_t c, uint64_t j) {
    uint64_t start_symbol = c;
    uint64_t code = t->code[c];
    uint32_t len = t->len[c];
    uint64_t result = j;
    for (int l = (int)len - 1; l >= 0; l--) {
        uint64_t counts;
        if ((code >> (t->L - 1 - (uint32_t)l)) & 1u) {
            start_symbol = o2_node_start(t, start_symbol, (uint32_t)l);
            counts = t->C[start_symbol];
            uint64_t start = lv_rank(&t->lv[l], 1, counts);
            result = lv_select(&t->lv[l], 1, start + result) + 1;
        } else {
            counts = t->C[start_symbol];
            uint64_t start = lv_rank(&t->lv[l], 0, counts);
            result = lv_select(&t->lv[l], 0, start + result) + 1;
        }
        result -= counts;
    }
    return result - 1;
}

void orc_o2_access(const orc_tree* t, const uint64_t* idx, uint64_t q, uint32_t* out) {
    for (uint64_t k = 0; k < q; k++) out[k] = idx[k] < t->n ? o2_access1(t, idx[k]) : UINT32_MAX;
}

void orc_o2_rank(const orc_tree* t, const uint32_t* c, const uint64_t* i, uint64_t q, uint64_t* out) {
    for (uint64_t k = 0; k < q; k++) {
        if (c[k] >= t->sigma || i[k] > t->n) out[k] = UINT64_MAX;
        else out[k] = o2_rank1(t, c[k], i[k]);
    }
}

void orc_o2_select(const orc_tree* t, const uint32_t* c, const uint64_t* j, uint64_t q, uint64_t* out) {
    for (uint64_t k = 0; k < q; k++) {
        if (c[k] >= t->sigma || j[k] == 0 || j[k] > t->C[c[k] + 1] - t->C[c[k]]) out[k] = UINT64_MAX;
        else out[k] = o2_select1(t, c[k], j[k]);
    }
}

/* The query loops above over nt threads, each taking a contiguous range of
 * the batch: kind 0 access (out uint32), 1 rank, 2 select (out uint64).     */
typedef struct {
    const orc_tree* t;
    int kind;
    const uint32_t* c;
    const uint64_t* arg;
    uint64_t a, b;
    void* out;
} orc_q_job;

static void* orc_q_run(void* p) {
    orc_q_job* j = (orc_q_job*)p;
    uint64_t q = j->b - j->a;
    if (j->kind == 0) orc_o2_access(j->t, j->arg + j->a, q, (uint32_t*)j->out + j->a);
    else if (j->kind == 1) orc_o2_rank(j->t, j->c + j->a, j->arg + j->a, q, (uint64_t*)j->out + j->a);
    else orc_o2_select(j->t, j->c + j->a, j->arg + j->a, q, (uint64_t*)j->out + j->a);
    return NULL;
}

void orc_o2_query_mt(const orc_tree* t, int kind, const uint32_t* c, const uint64_t* arg, uint64_t q, void* out,
                     int threads) {
    orc_q_job jobs[ORC_MAX_THREADS];
    const int nt = orc_threads(threads, q * 64);
    for (int i = 0; i < nt; i++) {
        jobs[i].t = t;
        jobs[i].kind = kind;
        jobs[i].c = c;
        jobs[i].arg = arg;
        jobs[i].out = out;
        orc_split(q, nt, i, &jobs[i].a, &jobs[i].b);
    }
    orc_run(orc_q_run, jobs, sizeof(jobs[0]), nt);
}

/* Number of threads orc_o2_build_mt and orc_o2_query_mt use by default. */
int orc_default_threads(void) { return orc_threads(0, (uint64_t)1 << 40); }
