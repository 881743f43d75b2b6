/*
 * serial_ct.c -- a plain serial Compact-Table propagator on the CPU.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY: the CPU bitset baseline that the
 * benchmark times beside the GPU library and the oracle, and a third opinion
 * in the CPU tests. It shares no code with the CUDA library.
 *
 * It follows the serial propagator of Sec. 3 and Algorithms 1-3 directly,
 * one propagation at a time on one host thread:
 *   - currTable is a reversible sparse bitset of 64-bit words: `index` lists
 *     the non-zero words in its first `limit` slots; a word that becomes zero
 *     is swapped to position limit-1 and limit shrinks (restoring limit
 *     restores the set);
 *   - updateTable (Algorithm 2) collects, for each variable whose domain
 *     shrank, the OR of the supports of its removed values (complemented) when
 *     |Delta| < |dom|, else the OR of the supports of its remaining values, and
 *     intersects currTable with it over the non-zero words;
 *   - filterDomains (Algorithm 3) checks each remaining value of each variable
 *     with more than one value: first its residue word, then the non-zero
 *     words in index order; a value without support is removed;
 *   - lastSizes of Algorithm 1 is kept as the last domains (bitsets), so that
 *     Delta is known exactly;
 *   - backtracking: every changed word is trailed once per level; a level
 *     stores the trail size, the limit and the last domains.
 * Domains use the library's layout: per variable ceil(size/32) uint32 words,
 * value lo+a at bit a%32 of word a/32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t trail_size;
    int32_t limit;
    uint32_t* last;  /* lastDom snapshot */
} sct_level;

typedef struct sct_table {
    int arity;
    int32_t* lo;
    int32_t* size;
    int32_t* nw;      /* 32-bit domain words per variable */
    int32_t* ld;      /* offset of each variable in the packed domains */
    int32_t* row0;    /* first supports row of each variable */
    int R, DW;
    int64_t t, W;     /* retained tuples, 64-bit words */
    uint64_t* sup;    /* [R][W] */
    uint64_t* curr;   /* [W] */
    int32_t* index;   /* [W] */
    int32_t limit;
    int32_t* residue; /* [R] */
    uint32_t* last;   /* [DW] */
    uint64_t* mask;   /* [W] scratch */
    uint64_t* tmp;    /* [W] scratch */
    int32_t* tw;      /* trail: word */
    uint64_t* tv;     /* trail: old value */
    int32_t tsize, tcap;
    int32_t* stamp;   /* [W] level at which the word was last trailed (+1) */
    sct_level* lev;
    int nlev, levcap;
    int failed;
} sct_table;

static int popc32(uint32_t x) { return __builtin_popcount(x); }

void sct_destroy(sct_table* T) {
    if (!T) return;
    free(T->lo); free(T->size); free(T->nw); free(T->ld); free(T->row0);
    free(T->sup); free(T->curr); free(T->index); free(T->residue); free(T->last);
    free(T->mask); free(T->tmp); free(T->tw); free(T->tv); free(T->stamp);
    for (int l = 0; l < T->levcap; ++l) free(T->lev[l].last);
    free(T->lev);
    free(T);
}

/* Build the table (Sec. 3 constructor). Returns NULL on bad input; *status
 * receives 0 (ok) or 1 (no tuple fits the initial domains). */
sct_table* sct_create(int arity, const int32_t* dom_lo, const int32_t* dom_size, const int32_t* tuples, int64_t t,
                      int* status) {
    sct_table* T = (sct_table*)calloc(1, sizeof(sct_table));
    if (!T) return NULL;
    T->arity = arity;
    T->lo = (int32_t*)malloc(sizeof(int32_t) * arity);
    T->size = (int32_t*)malloc(sizeof(int32_t) * arity);
    T->nw = (int32_t*)malloc(sizeof(int32_t) * arity);
    T->ld = (int32_t*)malloc(sizeof(int32_t) * arity);
    T->row0 = (int32_t*)malloc(sizeof(int32_t) * arity);
    for (int i = 0; i < arity; ++i) {
        T->lo[i] = dom_lo[i];
        T->size[i] = dom_size[i];
        T->nw[i] = (dom_size[i] + 31) / 32;
        T->ld[i] = T->DW;
        T->row0[i] = T->R;
        T->DW += T->nw[i];
        T->R += dom_size[i];
    }
    int64_t kept = 0;
    for (int64_t j = 0; j < t; ++j) {
        int ok = 1;
        for (int i = 0; i < arity && ok; ++i) {
            const int64_t off = (int64_t)tuples[j * arity + i] - dom_lo[i];
            ok = off >= 0 && off < dom_size[i];
        }
        kept += ok;
    }
    T->t = kept;
    T->W = (kept + 63) / 64;
    const int64_t W = T->W > 0 ? T->W : 1;
    T->sup = (uint64_t*)calloc((size_t)T->R * W, sizeof(uint64_t));
    T->curr = (uint64_t*)calloc(W, sizeof(uint64_t));
    T->index = (int32_t*)malloc(sizeof(int32_t) * W);
    T->residue = (int32_t*)calloc(T->R, sizeof(int32_t));
    T->last = (uint32_t*)calloc(T->DW, sizeof(uint32_t));
    T->mask = (uint64_t*)malloc(sizeof(uint64_t) * W);
    T->tmp = (uint64_t*)malloc(sizeof(uint64_t) * W);
    T->stamp = (int32_t*)calloc(W, sizeof(int32_t));
    if (!T->sup || !T->curr || !T->index || !T->residue || !T->last || !T->mask || !T->tmp || !T->stamp) {
        sct_destroy(T);
        return NULL;
    }
    int64_t jj = 0;
    for (int64_t j = 0; j < t; ++j) {
        int ok = 1;
        for (int i = 0; i < arity && ok; ++i) {
            const int64_t off = (int64_t)tuples[j * arity + i] - dom_lo[i];
            ok = off >= 0 && off < dom_size[i];
        }
        if (!ok) continue;
        for (int i = 0; i < arity; ++i) {
            const int r = T->row0[i] + (tuples[j * arity + i] - dom_lo[i]);
            T->sup[(size_t)r * W + (jj >> 6)] |= 1ull << (jj & 63);
        }
        T->curr[jj >> 6] |= 1ull << (jj & 63);
        ++jj;
    }
    T->limit = (int32_t)T->W;
    for (int64_t w = 0; w < T->W; ++w) T->index[w] = (int32_t)w;
    for (int r = 0; r < T->R; ++r) {
        for (int64_t w = 0; w < T->W; ++w) {
            if (T->sup[(size_t)r * W + w]) {
                T->residue[r] = (int32_t)w;
                break;
            }
        }
    }
    for (int i = 0; i < arity; ++i)
        for (int a = 0; a < dom_size[i]; ++a) T->last[T->ld[i] + a / 32] |= 1u << (a % 32);
    *status = kept == 0 ? 1 : 0;
    T->failed = kept == 0;
    return T;
}

static void trail_word(sct_table* T, int32_t w) {
    if (T->nlev == 0 || T->stamp[w] == T->nlev) return;
    if (T->tsize == T->tcap) {
        const int32_t cap = T->tcap ? 2 * T->tcap : 1024;
        T->tw = (int32_t*)realloc(T->tw, sizeof(int32_t) * cap);
        T->tv = (uint64_t*)realloc(T->tv, sizeof(uint64_t) * cap);
        T->tcap = cap;
    }
    T->tw[T->tsize] = w;
    T->tv[T->tsize] = T->curr[w];
    T->tsize++;
    T->stamp[w] = T->nlev;
}

/* Algorithms 1-3 on the packed domains (in/out). Returns 0 (ok), 1 (fail),
 * -4 (a domain grew since the last call) or -1 (bad state). */
int sct_propagate(sct_table* T, uint32_t* dom) {
    if (!T || T->failed) return T && T->t == 0 ? 1 : -1;
    const int64_t W = T->W;
    /* Algorithm 1, lines 1-3: s_val (domains that shrank) and s_sup. */
    for (int i = 0; i < T->arity; ++i)
        for (int q = 0; q < T->nw[i]; ++q)
            if (dom[T->ld[i] + q] & ~T->last[T->ld[i] + q]) return -4;
    for (int i = 0; i < T->arity; ++i) {
        int nd = 0, ndel = 0;
        for (int q = 0; q < T->nw[i]; ++q) {
            const uint32_t d = dom[T->ld[i] + q], l = T->last[T->ld[i] + q];
            nd += popc32(d);
            ndel += popc32(l & ~d);
        }
        if (nd == 0) {
            T->failed = 1;
            return 1;
        }
        if (ndel == 0) continue;
        /* Algorithm 2: the mask of variable i over the non-zero words. */
        for (int k = 0; k < T->limit; ++k) T->mask[T->index[k]] = 0;
        const int delta = ndel < nd;
        for (int q = 0; q < T->nw[i]; ++q) {
            const uint32_t d = dom[T->ld[i] + q], l = T->last[T->ld[i] + q];
            uint32_t bits = delta ? (l & ~d) : d;
            while (bits) {
                const int b = __builtin_ctz(bits);
                bits &= bits - 1;
                const uint64_t* row = T->sup + (size_t)(T->row0[i] + q * 32 + b) * (W > 0 ? W : 1);
                for (int k = 0; k < T->limit; ++k) T->mask[T->index[k]] |= row[T->index[k]];
            }
        }
        for (int k = T->limit - 1; k >= 0; --k) {
            const int32_t w = T->index[k];
            const uint64_t m = delta ? ~T->mask[w] : T->mask[w];
            const uint64_t nv = T->curr[w] & m;
            if (nv != T->curr[w]) {
                trail_word(T, w);
                T->curr[w] = nv;
            }
            if (nv == 0) {
                /* swap with the last non-zero word */
                T->index[k] = T->index[T->limit - 1];
                T->index[T->limit - 1] = w;
                T->limit--;
            }
        }
        if (T->limit == 0) break;
    }
    /* Algorithm 1, line 5 */
    if (T->limit == 0) {
        T->failed = 1;
        return 1;
    }
    /* Algorithm 3 (with residues): s_sup = variables with more than one value. */
    for (int i = 0; i < T->arity; ++i) {
        int nd = 0;
        for (int q = 0; q < T->nw[i]; ++q) nd += popc32(dom[T->ld[i] + q]);
        if (nd > 1) {
            for (int q = 0; q < T->nw[i]; ++q) {
                uint32_t bits = dom[T->ld[i] + q];
                while (bits) {
                    const int b = __builtin_ctz(bits);
                    bits &= bits - 1;
                    const int r = T->row0[i] + q * 32 + b;
                    const uint64_t* row = T->sup + (size_t)r * W;
                    const int32_t res = T->residue[r];
                    if (T->curr[res] & row[res]) continue;
                    int found = -1;
                    for (int k = 0; k < T->limit; ++k) {
                        const int32_t w = T->index[k];
                        if (T->curr[w] & row[w]) {
                            found = w;
                            break;
                        }
                    }
                    if (found >= 0) {
                        T->residue[r] = found;
                    } else {
                        dom[T->ld[i] + q] &= ~(1u << b);
                    }
                }
            }
        }
        /* lastSizes := the filtered domain */
        for (int q = 0; q < T->nw[i]; ++q) T->last[T->ld[i] + q] = dom[T->ld[i] + q];
    }
    return 0;
}

int sct_save(sct_table* T) {
    if (T->nlev == T->levcap) {
        const int cap = T->levcap ? 2 * T->levcap : 16;
        T->lev = (sct_level*)realloc(T->lev, sizeof(sct_level) * cap);
        for (int l = T->levcap; l < cap; ++l) T->lev[l].last = (uint32_t*)malloc(sizeof(uint32_t) * (T->DW ? T->DW : 1));
        T->levcap = cap;
    }
    sct_level* L = &T->lev[T->nlev];
    L->trail_size = T->tsize;
    L->limit = T->limit;
    memcpy(L->last, T->last, sizeof(uint32_t) * T->DW);
    T->nlev++;
    return T->nlev - 1;
}

/* Back to the state at sct_save() == level; drops that level and those above. */
int sct_restore(sct_table* T, int level) {
    if (level < 0 || level >= T->nlev) return -6;
    sct_level* L = &T->lev[level];
    for (int32_t p = T->tsize - 1; p >= L->trail_size; --p) {
        T->curr[T->tw[p]] = T->tv[p];
        T->stamp[T->tw[p]] = 0;
    }
    T->tsize = L->trail_size;
    T->limit = L->limit;
    memcpy(T->last, L->last, sizeof(uint32_t) * T->DW);
    T->nlev = level;
    T->failed = T->t == 0;
    return 0;
}

/* currTable as 32-bit words (tuple j at bit j%32 of word j/32). */
void sct_currtable32(const sct_table* T, uint32_t* out) {
    const int64_t W32 = (T->t + 31) / 32;
    for (int64_t w = 0; w < W32; ++w) out[w] = (uint32_t)(T->curr[w >> 1] >> (32 * (w & 1)));
}

int64_t sct_live_words(const sct_table* T) { return T->limit; }
