/*
 * CPU oracle for DFA state equivalence (arXiv 2410.22764, "An Evaluation of Massively
 * Parallel Algorithms for DFA Minimization").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential statement of what the
 * GPU library computes.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Conventions shared with the library's public contract (they are part of the problem
 * statement, not of any implementation):
 *   - states are 0..n-1 and letters 0..k-1 (Sec. 2 "Representation", read as 0-based);
 *   - delta is state-major: delta[s*k + a] = delta(s, a);
 *   - accept is a bitmap, LSB first: state s is accepting iff (accept[s>>5] >> (s&31)) & 1;
 *   - the result is the coarsest partition of ALL states that refines {F, Q\F} and is stable
 *     under delta (Sec. 2, problem statement: unreachable states are not removed);
 *   - block labels are canonical: a block's id is the number of blocks whose smallest state
 *     is smaller than its own smallest state (first-occurrence order over s = 0..n-1).
 *
 * Functions:
 *   oracle_canonical   canonical relabelling of any labelling
 *   oracle_moore       Moore refinement written as the steps of Alg. sortPR (Sec. 3.3)
 *   oracle_hopcroft    Hopcroft's splitter-worklist refinement (Sec. 1, [Hopcroft 1971])
 *   oracle_tablefill   pairwise marking: the sequential meaning of Alg. 1 "trans" (Sec. 3.1)
 *   oracle_closure     the per-letter partial transitive closure of Alg. transPR (Sec. 3.4)
 *   oracle_naive       leader-election refinement, the steps of Alg. 2 naivePR (Sec. 3.2)
 *   oracle_reachable   states reachable from q0, order-preserving renumbering (Sec. 2)
 *   oracle_quotient    the quotient automaton of a stable partition (Sec. 2)
 *   oracle_check_stable  property check: refines {F, Q\F} and is stable under delta
 *
 * Every routine returns 0 on success and a negative value on bad arguments or allocation
 * failure.  Every routine is single-threaded.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EARG (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ENOCONVERGE (-3)

static int is_accepting(const uint32_t *accept, int64_t s)
{
    return (int)((accept[s >> 5] >> (s & 31)) & 1u);
}

static int check_delta(int32_t n, int32_t k, const int32_t *delta)
{
    int64_t total = (int64_t)n * (int64_t)k;
    for (int64_t i = 0; i < total; i++)
        if (delta[i] < 0 || delta[i] >= n)
            return ORACLE_EARG;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------
 * Canonical labels: scan s = 0..n-1 and give each label a fresh id the first time it is seen.
 * The id of a block is then the rank of its smallest state among the blocks' smallest states.
 * Input labels must lie in [0, n).  Writes out[n] and returns the number of blocks in *count.
 * ------------------------------------------------------------------------------------------ */
int oracle_canonical(int32_t n, const int32_t *label, int32_t *out, int32_t *count)
{
    if (n < 0 || (n > 0 && (!label || !out)))
        return ORACLE_EARG;
    int32_t *map = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!map)
        return ORACLE_ENOMEM;
    for (int32_t i = 0; i < n; i++)
        map[i] = -1;
    int32_t next = 0;
    for (int32_t s = 0; s < n; s++) {
        int32_t l = label[s];
        if (l < 0 || l >= n) {
            free(map);
            return ORACLE_EARG;
        }
        if (map[l] < 0)
            map[l] = next++;
        out[s] = map[l];
    }
    free(map);
    if (count)
        *count = next;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------
 * Moore refinement, written as the steps of Alg. sortPR (Sec. 3.3):
 *   init:   block[q] := (q in F ? 0 : 1); state[q] := q
 *   repeat: signature[q][a] := block[delta(q, a)]
 *           sort state[] with COMPARE (block first, then signature letters in order)
 *           new_block[i] := ARE_NEQ(state[i], state[i-1]) for i > 0; new_block[0] := 0
 *           inclusive scan of new_block
 *           block[state[i]] := new_block[i]
 *   until the number of blocks did not change.
 * Readings where the paper's listing is loose (each is also stated in the design notes):
 *   - the initial count is the number of non-empty parts of {F, Q\F} (1 or 2), not a fixed 2;
 *   - the loop also stops when every block is a singleton (count == n); with that rule the
 *     pass counts are n-2 on the cyclic Fibonacci automata (Sec. 4.2 text) and n-1 on the
 *     bit-splitters B_n (Table 2);
 *   - *passes counts executed signature rounds; it is 0 when {F, Q\F} is already discrete;
 *   - the ids inside the loop are sorted-order ids; the result is relabelled canonically.
 * The sort is a stable merge sort on state indices with COMPARE as the order.
 * max_passes <= 0 means no cap.  Returns ORACLE_ENOCONVERGE if the cap is reached first; the
 * partition after the capped passes is still written (canonically) to out_block.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t k;
    const int32_t *block;
    const int32_t *signature; /* [n*k] */
} moore_ctx;

/* COMPARE of Alg. sortPR as a three-way comparison: block first, then letters in order. */
static int moore_compare(const moore_ctx *c, int32_t q1, int32_t q2)
{
    if (c->block[q1] != c->block[q2])
        return c->block[q1] < c->block[q2] ? -1 : 1;
    const int32_t *s1 = c->signature + (int64_t)q1 * c->k;
    const int32_t *s2 = c->signature + (int64_t)q2 * c->k;
    for (int32_t a = 0; a < c->k; a++)
        if (s1[a] != s2[a])
            return s1[a] < s2[a] ? -1 : 1;
    return 0;
}

static void merge_sort(const moore_ctx *c, int32_t *v, int32_t *tmp, int32_t n)
{
    for (int32_t width = 1; width < n; width *= 2) {
        for (int32_t lo = 0; lo < n; lo += 2 * width) {
            int32_t mid = lo + width < n ? lo + width : n;
            int32_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int32_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi)
                tmp[o++] = (moore_compare(c, v[j], v[i]) < 0) ? v[j++] : v[i++];
            while (i < mid)
                tmp[o++] = v[i++];
            while (j < hi)
                tmp[o++] = v[j++];
        }
        memcpy(v, tmp, sizeof(int32_t) * (size_t)n);
    }
}

int oracle_moore(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                 int32_t max_passes, int32_t *out_block, int32_t *nblocks, int32_t *passes)
{
    if (n < 1 || k < 0 || (k > 0 && !delta) || !accept || !out_block)
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    size_t nn = (size_t)n;
    int32_t *block = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *state = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *new_block = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *signature = (int32_t *)malloc(sizeof(int32_t) * (nn * (size_t)k + 1));
    if (!block || !state || !tmp || !new_block || !signature) {
        free(block); free(state); free(tmp); free(new_block); free(signature);
        return ORACLE_ENOMEM;
    }
    /* init: accepting -> 0, rejecting -> 1 */
    int have_f = 0, have_nf = 0;
    for (int32_t q = 0; q < n; q++) {
        int f = is_accepting(accept, q);
        block[q] = f ? 0 : 1;
        have_f |= f;
        have_nf |= !f;
        state[q] = q;
    }
    if (n == 1)
        block[0] = 0; /* the listing's label 1 would fall outside [0, n) */
    int32_t num_blocks = have_f + have_nf;
    int32_t count = num_blocks;
    int32_t p = 0;
    int rc = ORACLE_OK;
    moore_ctx ctx = {k, block, signature};
    while (count < n) {
        if (max_passes > 0 && p >= max_passes) {
            rc = ORACLE_ENOCONVERGE;
            break;
        }
        num_blocks = count;
        for (int32_t q = 0; q < n; q++)
            for (int32_t a = 0; a < k; a++)
                signature[(int64_t)q * k + a] = block[delta[(int64_t)q * k + a]];
        merge_sort(&ctx, state, tmp, n);
        /* adjacent difference with ARE_NEQ, first entry 0, then inclusive scan */
        new_block[0] = 0;
        for (int32_t i = 1; i < n; i++)
            new_block[i] = moore_compare(&ctx, state[i], state[i - 1]) != 0 ? 1 : 0;
        for (int32_t i = 1; i < n; i++)
            new_block[i] += new_block[i - 1];
        for (int32_t i = 0; i < n; i++)
            block[state[i]] = new_block[i];
        count = new_block[n - 1] + 1;
        p++;
        if (count == num_blocks)
            break;
    }
    int32_t c = 0;
    int rc2 = oracle_canonical(n, block, out_block, &c);
    if (rc == ORACLE_OK)
        rc = rc2;
    if (nblocks)
        *nblocks = c;
    if (passes)
        *passes = p;
    free(block); free(state); free(tmp); free(new_block); free(signature);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Hopcroft's algorithm.  The partition is kept as an array of states in which every block is a
 * contiguous range; marking moves a state to the front part of its block's range.  A worklist
 * holds (block, letter) splitters.  Initially it holds (smaller of F and Q\F, a) for every a.
 * Processing splitter (C, a) marks every p with delta(p, a) in C; every block with some but not
 * all states marked is split into its marked part and the rest; for every letter b the worklist
 * then receives the new block if (old block, b) is pending, and the smaller half otherwise.
 * ------------------------------------------------------------------------------------------ */
int oracle_hopcroft(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                    int32_t *out_block, int32_t *nblocks)
{
    if (n < 1 || k < 0 || (k > 0 && !delta) || !accept || !out_block)
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    size_t nn = (size_t)n, nk = (size_t)n * (size_t)k;
    int32_t *elems = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *blk = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *first = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *end = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *mid = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *splitter = (int32_t *)malloc(sizeof(int32_t) * nn);
    /* inverse transitions, one CSR per letter: pred_off[a*(n+1) + q] .. */
    int64_t *pred_off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)k * (nn + 1) + 1));
    int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (nk + 1));
    uint8_t *pending = (uint8_t *)calloc(nk + 1, 1); /* pending[b*k + a] */
    /* worklist as a stack of (block, letter); every (block, letter) is on it at most once */
    int64_t *work = (int64_t *)malloc(sizeof(int64_t) * (nk + 1));
    if (!elems || !loc || !blk || !first || !end || !mid || !touched || !splitter ||
        !pred_off || !pred || !pending || !work) {
        free(elems); free(loc); free(blk); free(first); free(end); free(mid); free(touched);
        free(splitter); free(pred_off); free(pred); free(pending); free(work);
        return ORACLE_ENOMEM;
    }
    for (int32_t a = 0; a < k; a++) {
        int64_t *off = pred_off + (size_t)a * (nn + 1);
        memset(off, 0, sizeof(int64_t) * (nn + 1));
        for (int32_t q = 0; q < n; q++)
            off[delta[(int64_t)q * k + a] + 1]++;
        for (int32_t q = 0; q < n; q++)
            off[q + 1] += off[q];
    }
    for (int32_t a = 0; a < k; a++) {
        int64_t *off = pred_off + (size_t)a * (nn + 1);
        int32_t *p = pred + (size_t)a * nn;
        /* fill in increasing order of the source state, using end[] as a cursor */
        for (int32_t q = 0; q < n; q++)
            end[q] = 0;
        for (int32_t q = 0; q < n; q++) {
            int32_t t = delta[(int64_t)q * k + a];
            p[off[t] + end[t]++] = q;
        }
    }
    /* initial partition {F, Q\F}: accepting states first */
    int32_t nf = 0;
    for (int32_t q = 0; q < n; q++)
        if (is_accepting(accept, q))
            nf++;
    int32_t fi = 0, ri = nf;
    for (int32_t q = 0; q < n; q++) {
        int32_t i = is_accepting(accept, q) ? fi++ : ri++;
        elems[i] = q;
        loc[q] = i;
    }
    int32_t nb = 0;
    int32_t bF = -1, bN = -1;
    if (nf > 0) {
        bF = nb++;
        first[bF] = 0; end[bF] = nf; mid[bF] = 0;
    }
    if (nf < n) {
        bN = nb++;
        first[bN] = nf; end[bN] = n; mid[bN] = nf;
    }
    for (int32_t q = 0; q < n; q++)
        blk[q] = is_accepting(accept, q) ? bF : bN;
    int64_t wtop = 0;
    if (bF >= 0 && bN >= 0) {
        int32_t smaller = (nf <= n - nf) ? bF : bN;
        for (int32_t a = 0; a < k; a++) {
            work[wtop++] = (int64_t)smaller * k + a;
            pending[(size_t)smaller * k + a] = 1;
        }
    }
    while (wtop > 0) {
        int64_t item = work[--wtop];
        int32_t C = (int32_t)(item / k), a = (int32_t)(item % k);
        pending[(size_t)C * k + a] = 0;
        /* copy the splitter's states first: marking reorders states inside blocks */
        int32_t csize = end[C] - first[C];
        memcpy(splitter, elems + first[C], sizeof(int32_t) * (size_t)csize);
        int32_t ntouched = 0;
        const int64_t *off = pred_off + (size_t)a * (nn + 1);
        const int32_t *pa = pred + (size_t)a * nn;
        for (int32_t ci = 0; ci < csize; ci++) {
            int32_t q = splitter[ci];
            for (int64_t e = off[q]; e < off[q + 1]; e++) {
                int32_t p = pa[e];
                int32_t b = blk[p];
                int32_t i = loc[p];
                if (i < mid[b])
                    continue; /* already marked */
                if (mid[b] == first[b])
                    touched[ntouched++] = b;
                int32_t j = mid[b]++;
                int32_t other = elems[j];
                elems[j] = p; loc[p] = j;
                elems[i] = other; loc[other] = i;
            }
        }
        for (int32_t t = 0; t < ntouched; t++) {
            int32_t b = touched[t];
            if (mid[b] == end[b]) { /* every state marked: no split */
                mid[b] = first[b];
                continue;
            }
            int32_t nbk = nb++;
            first[nbk] = first[b];
            end[nbk] = mid[b];
            mid[nbk] = first[nbk];
            first[b] = mid[b];
            mid[b] = first[b];
            for (int32_t i = first[nbk]; i < end[nbk]; i++)
                blk[elems[i]] = nbk;
            int32_t size_new = end[nbk] - first[nbk], size_old = end[b] - first[b];
            for (int32_t bb = 0; bb < k; bb++) {
                if (pending[(size_t)b * k + bb]) {
                    work[wtop++] = (int64_t)nbk * k + bb;
                    pending[(size_t)nbk * k + bb] = 1;
                } else {
                    int32_t add = (size_new <= size_old) ? nbk : b;
                    work[wtop++] = (int64_t)add * k + bb;
                    pending[(size_t)add * k + bb] = 1;
                }
            }
        }
    }
    int32_t c = 0;
    int rc = oracle_canonical(n, blk, out_block, &c);
    if (nblocks)
        *nblocks = c;
    free(elems); free(loc); free(blk); free(first); free(end); free(mid); free(touched);
    free(splitter); free(pred_off); free(pred); free(pending); free(work);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Pairwise marking (table filling), the sequential meaning of Alg. 1 "trans" (Sec. 3.1):
 * pair (p, q) is apart if exactly one of p, q is accepting, or if some letter leads to an
 * apart pair.  Rounds are synchronous: round r marks the pairs whose shortest distinguishing
 * word has length exactly r, so *rounds is the largest such length (the distinguishing depth).
 * p and q are equivalent iff the pair is never marked.  Memory is n*n bytes: keep n small.
 * ------------------------------------------------------------------------------------------ */
int oracle_tablefill(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                     int32_t *out_block, int32_t *nblocks, int32_t *rounds)
{
    if (n < 1 || n > 20000 || k < 0 || (k > 0 && !delta) || !accept || !out_block)
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    size_t nn = (size_t)n;
    uint8_t *apart = (uint8_t *)malloc(nn * nn);
    uint8_t *next = (uint8_t *)malloc(nn * nn);
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!apart || !next || !label) {
        free(apart); free(next); free(label);
        return ORACLE_ENOMEM;
    }
    for (int32_t p = 0; p < n; p++)
        for (int32_t q = 0; q < n; q++)
            apart[(size_t)p * nn + q] = is_accepting(accept, p) != is_accepting(accept, q);
    int32_t r = 0;
    for (;;) {
        memcpy(next, apart, nn * nn);
        int changed = 0;
        for (int32_t p = 0; p < n; p++)
            for (int32_t q = p + 1; q < n; q++) {
                if (apart[(size_t)p * nn + q])
                    continue;
                for (int32_t a = 0; a < k; a++) {
                    int32_t dp = delta[(int64_t)p * k + a], dq = delta[(int64_t)q * k + a];
                    if (apart[(size_t)dp * nn + dq]) {
                        next[(size_t)p * nn + q] = next[(size_t)q * nn + p] = 1;
                        changed = 1;
                        break;
                    }
                }
            }
        if (!changed)
            break;
        memcpy(apart, next, nn * nn);
        r++;
    }
    /* label each state by the smallest state it is not apart from */
    for (int32_t s = 0; s < n; s++) {
        label[s] = s;
        for (int32_t t = 0; t < s; t++)
            if (!apart[(size_t)s * nn + t]) {
                label[s] = label[t];
                break;
            }
    }
    int32_t c = 0;
    int rc = oracle_canonical(n, label, out_block, &c);
    if (nblocks)
        *nblocks = c;
    if (rounds)
        *rounds = r;
    free(apart); free(next); free(label);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * Partial transitive closure of Alg. transPR (Sec. 3.4): the alphabet grows to the words
 * a^(2^i) for every letter a and i = 0..floor(log2 n); the transition on a^(2^i) is the
 * transition on a^(2^(i-1)) taken twice.  Level i of letter a is written as one column of n
 * states, letter-major: out[(a*levels + i)*n + q] = delta^T(q, a^(2^i)), with
 * levels = floor(log2 n) + 1 (so level 0 is delta itself).  Level i reads only level i-1.
 * ------------------------------------------------------------------------------------------ */
int32_t oracle_closure_levels(int32_t n)
{
    if (n < 1)
        return 0;
    int32_t l = 0;
    while (((int64_t)1 << (l + 1)) <= (int64_t)n)
        l++;
    return l + 1;
}

int oracle_closure(int32_t n, int32_t k, const int32_t *delta, int32_t *out)
{
    if (n < 1 || k < 0 || (k > 0 && (!delta || !out)))
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    int32_t levels = oracle_closure_levels(n);
    size_t nn = (size_t)n;
    for (int32_t a = 0; a < k; a++) {
        int32_t *col0 = out + ((size_t)a * levels) * nn;
        for (int32_t q = 0; q < n; q++)
            col0[q] = delta[(int64_t)q * k + a];
        for (int32_t i = 1; i < levels; i++) {
            const int32_t *prev = out + ((size_t)a * levels + (size_t)(i - 1)) * nn;
            int32_t *cur = out + ((size_t)a * levels + (size_t)i) * nn;
            for (int32_t q = 0; q < n; q++)
                cur[q] = prev[prev[q]];
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------
 * Property check for any size: the labelling refines {F, Q\F} and is stable under delta
 * (states with one label have successors with one label, per letter).  Labels in [0, n).
 * Returns 1 if both hold, 0 if not, negative on bad arguments.  A stable partition refining
 * {F, Q\F} is a congruence, so it is at least as fine as the coarsest one; equality with the
 * coarsest partition additionally needs the block count from an oracle.
 * ------------------------------------------------------------------------------------------ */
int oracle_check_stable(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                        const int32_t *label)
{
    if (n < 1 || k < 0 || (k > 0 && !delta) || !accept || !label)
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    size_t nn = (size_t)n;
    int32_t *rep = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!rep)
        return ORACLE_ENOMEM;
    for (int32_t i = 0; i < n; i++)
        rep[i] = -1;
    int ok = 1;
    for (int32_t s = 0; s < n && ok; s++) {
        int32_t l = label[s];
        if (l < 0 || l >= n) {
            ok = 0;
            break;
        }
        if (rep[l] < 0) {
            rep[l] = s;
            continue;
        }
        int32_t t = rep[l];
        if (is_accepting(accept, s) != is_accepting(accept, t))
            ok = 0;
        for (int32_t a = 0; a < k && ok; a++)
            if (label[delta[(int64_t)s * k + a]] != label[delta[(int64_t)t * k + a]])
                ok = 0;
    }
    free(rep);
    return ok;
}

/* ------------------------------------------------------------------------------------------
 * Leader-election refinement, the steps of Alg. 2 naivePR (Sec. 3.2):
 *   block[q] := (q in F ? q_f : q_n)                      initial leaders
 *   while not stable:
 *     stable := true
 *     for all (q, a): if block[delta(q,a)] != block[delta(block[q], a)]:
 *         new_leader[block[q]] := q                         leader election
 *     for all (q, a): if block[delta(q,a)] != block[delta(block[q], a)]:
 *         block[q] := new_leader[block[q]]; stable := false split from the leader
 * Readings (also in the design notes): the initial leaders are the smallest accepting and the
 * smallest rejecting state; of the concurrent writes of one election the smallest q wins
 * (the listing lets any one win); each parallel loop reads block[] as it was before the loop
 * (synchronous PRAM step).  *iters counts executed while-iterations, the final one that finds
 * nothing to split included.  max_iters <= 0 means no cap.
 * ------------------------------------------------------------------------------------------ */
int oracle_naive(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                 int32_t max_iters, int32_t *out_block, int32_t *nblocks, int32_t *iters)
{
    if (n < 1 || k < 0 || (k > 0 && !delta) || !accept || !out_block)
        return ORACLE_EARG;
    if (check_delta(n, k, delta) != ORACLE_OK)
        return ORACLE_EARG;
    size_t nn = (size_t)n;
    int32_t *block = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *new_leader = (int32_t *)malloc(sizeof(int32_t) * nn);
    uint8_t *differs = (uint8_t *)malloc(nn);
    if (!block || !next || !new_leader || !differs) {
        free(block); free(next); free(new_leader); free(differs);
        return ORACLE_ENOMEM;
    }
    int32_t qf = -1, qn = -1;
    for (int32_t q = 0; q < n; q++) {
        if (is_accepting(accept, q)) { if (qf < 0) qf = q; }
        else if (qn < 0) qn = q;
    }
    for (int32_t q = 0; q < n; q++)
        block[q] = is_accepting(accept, q) ? qf : qn;
    int32_t it = 0;
    int rc = ORACLE_OK;
    for (;;) {
        if (max_iters > 0 && it >= max_iters) {
            rc = ORACLE_ENOCONVERGE;
            break;
        }
        it++;
        int stable = 1;
        for (int32_t q = 0; q < n; q++) {
            differs[q] = 0;
            new_leader[q] = -1;
        }
        /* election: reads block[] only */
        for (int32_t q = 0; q < n; q++)
            for (int32_t a = 0; a < k; a++) {
                int32_t l = block[q];
                if (block[delta[(int64_t)q * k + a]] != block[delta[(int64_t)l * k + a]]) {
                    differs[q] = 1;
                    if (new_leader[l] < 0 || q < new_leader[l])
                        new_leader[l] = q;
                }
            }
        /* split: every test reads the block[] of before the loop, then the writes apply */
        for (int32_t q = 0; q < n; q++)
            next[q] = differs[q] ? new_leader[block[q]] : block[q];
        for (int32_t q = 0; q < n; q++) {
            if (next[q] != block[q])
                stable = 0;
            block[q] = next[q];
        }
        if (stable)
            break;
    }
    int32_t c = 0;
    int rc2 = oracle_canonical(n, block, out_block, &c);
    if (rc == ORACLE_OK)
        rc = rc2;
    if (nblocks)
        *nblocks = c;
    if (iters)
        *iters = it;
    free(block); free(next); free(new_leader); free(differs);
    return rc;
}

/*
 * Reachable states (Sec. 2: minimization deletes the states that no word leads to from q0).
 * Plain breadth-first search from q0 with a FIFO queue.  out_newid[s] is the rank of s among
 * the reachable states in increasing state order (an order-preserving renumbering), or -1;
 * *count is the number of reachable states.
 */
int oracle_reachable(int32_t n, int32_t k, const int32_t *delta, int32_t q0, int32_t *out_newid,
                     int32_t *count)
{
    if (n < 1 || k < 0 || q0 < 0 || q0 >= n || !out_newid || !count || (k > 0 && !delta))
        return ORACLE_EARG;
    if (check_delta(n, k, delta)) return ORACLE_EARG;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *seen = (char *)calloc((size_t)n, 1);
    if (!queue || !seen) { free(queue); free(seen); return ORACLE_ENOMEM; }
    int32_t head = 0, tail = 0;
    queue[tail++] = q0;
    seen[q0] = 1;
    while (head < tail) {
        const int32_t s = queue[head++];
        for (int32_t a = 0; a < k; ++a) {
            const int32_t t = delta[(int64_t)s * k + a];
            if (!seen[t]) { seen[t] = 1; queue[tail++] = t; }
        }
    }
    int32_t c = 0;
    for (int32_t s = 0; s < n; ++s) out_newid[s] = seen[s] ? c++ : -1;
    *count = c;
    free(queue);
    free(seen);
    return ORACLE_OK;
}

/*
 * Quotient automaton A/~ (Sec. 2: merging equivalent states into one): given a partition
 * `block` of the states into nblocks classes, each stable under delta and refining {F, Q\F},
 * the class B goes to class block[delta(s, a)] on letter a for any s in B (stability makes the
 * choice irrelevant; the smallest state of B is used), B accepts iff its states do, and the
 * initial class is block[q0].  out_delta is [nblocks][k] state-major; out_accept a bitmap.
 */
int oracle_quotient(int32_t n, int32_t k, const int32_t *delta, const uint32_t *accept,
                    const int32_t *block, int32_t nblocks, int32_t q0, int32_t *out_delta,
                    uint32_t *out_accept, int32_t *out_q0)
{
    if (n < 1 || k < 0 || nblocks < 1 || nblocks > n || q0 < 0 || q0 >= n || !accept ||
        !block || !out_accept || !out_q0 || (k > 0 && (!delta || !out_delta)))
        return ORACLE_EARG;
    int32_t *rep = (int32_t *)malloc(sizeof(int32_t) * (size_t)nblocks);
    if (!rep) return ORACLE_ENOMEM;
    for (int32_t b = 0; b < nblocks; ++b) rep[b] = -1;
    for (int32_t s = n - 1; s >= 0; --s) {
        if (block[s] < 0 || block[s] >= nblocks) { free(rep); return ORACLE_EARG; }
        rep[block[s]] = s;
    }
    for (int32_t b = 0; b < nblocks; ++b)
        if (rep[b] < 0) { free(rep); return ORACLE_EARG; }
    memset(out_accept, 0, sizeof(uint32_t) * (size_t)((nblocks + 31) / 32));
    for (int32_t b = 0; b < nblocks; ++b) {
        for (int32_t a = 0; a < k; ++a)
            out_delta[(int64_t)b * k + a] = block[delta[(int64_t)rep[b] * k + a]];
        if (is_accepting(accept, rep[b])) out_accept[b >> 5] |= 1u << (b & 31);
    }
    *out_q0 = block[q0];
    free(rep);
    return ORACLE_OK;
}
