/*
 * oracle.c -- plain, slow, single-purpose CPU statement of the hot path of
 * PLAST (Nguyen & Lavenier, "Fine-grained parallelization of similarity
 * search between protein sequences", INRIA RR-6513, 2008).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; it exists so the CUDA library can be checked against an
 * independent statement of the method.  It shares no source, table or
 * helper with the CUDA library: the substitution matrix, the subset-seed
 * classes and the genetic code below are transcribed here on their own.
 *
 * Every function follows the paper's steps in the paper's order, with no
 * blocking, packing or reordering.  Where the paper leaves a value open the
 * reading used is stated at the function.  The functions and the pins that
 * check them (tests/test_oracle_*.py):
 *   blosum62 / score ............ invariants + Karlin-Altschul lambda
 *   seed_class / seed_key ....... Section 3.3.1 example and class counts
 *   index ....................... brute-force enumeration of words
 *   ungapped_pair ............... identity closed form, brute force, symmetry
 *   filter_pair ................. bound U <= F, identity closed form, worked
 *                                 example, brute force
 *   gapped_side / small_gapped .. band-0 reduction, Smith-Waterman bound and
 *                                 equality, single-gap closed form, symmetry
 *   translate6 .................. genetic-code degeneracy, back-translation
 *   smith_waterman .............. textbook cases worked by hand
 *
 * Alphabet (a reading: the paper gives no encoding): protein codes 0..19 are
 * A R N D C Q E G H I L K M F P S T W Y V, code 20 is the stop '*' that only
 * translated banks contain.  Nucleotides are A C G T = 0 1 2 3.
 *
 * Build: gcc -O2 -shared -fPIC -pthread oracle.c -o liboracle.so
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NAA 20
#define STOP 20
#define NKEYS 8800
#define NEG_INF (-1000000)

/* ------------------------------------------------------------------------
 * BLOSUM62 (Henikoff & Henikoff, PNAS 1992), half-bit units, in the order
 * A R N D C Q E G H I L K M F P S T W Y V *.  The stop row is -4 against
 * every residue and +1 against itself, as in the NCBI distribution.
 * Section 3.3.3 scores the ungapped extension with a substitution matrix;
 * the evaluation (Annex 1/2) uses BLOSUM62 as BLAST does by default.
 * ---------------------------------------------------------------------- */
static const int8_t B62[21][21] = {
    /*        A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V   * */
    /* A */ { 4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0, -4},
    /* R */ {-1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3, -4},
    /* N */ {-2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3, -4},
    /* D */ {-2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3, -4},
    /* C */ { 0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1, -4},
    /* Q */ {-1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2, -4},
    /* E */ {-1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2, -4},
    /* G */ { 0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3, -4},
    /* H */ {-2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3, -4},
    /* I */ {-1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3, -4},
    /* L */ {-1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1, -4},
    /* K */ {-1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2, -4},
    /* M */ {-1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1, -4},
    /* F */ {-2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1, -4},
    /* P */ {-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2, -4},
    /* S */ { 1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2, -4},
    /* T */ { 0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0, -4},
    /* W */ {-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3, -4},
    /* Y */ {-2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1, -4},
    /* V */ { 0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4, -4},
    /* * */ {-4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4,  1},
};

int oracle_score(int a, int b) { return B62[a][b]; }

/* ------------------------------------------------------------------------
 * Subset seed of Section 3.3.1 (W = 4 positions).
 *   position 1 and 4: every amino acid is its own class (20 classes).  The
 *     printed list omits I; read as a typo, I is its own class.
 *   position 2: c = {C,F,Y,W,M,L,I,V} and g = {G,P,A,T,S,N,H,Q,E,D,R,K}.
 *   position 3: A, C, f, G, i = {I,V}, m = {M,L}, n = {N,H}, P,
 *     q = {Q,E,D}, r = {R,K}, t = {T,S}.  The printed f = {F,Y,E} puts E in
 *     two classes and W in none; read as f = {F,Y,W} (11 classes).
 * Class numbers: positions 1 and 4 use the residue code; position 2 is
 * c = 0, g = 1; position 3 numbers its classes in the printed order
 * A=0 C=1 f=2 G=3 i=4 m=5 n=6 P=7 q=8 r=9 t=10.
 * Key = ((c1 * 2 + c2) * 11 + c3) * 20 + c4, so keys run over 0..8799.
 * ---------------------------------------------------------------------- */
static int class_pos2(int aa) {
  /* c = {C,F,Y,W,M,L,I,V} */
  switch (aa) {
    case 4: case 13: case 18: case 17: case 12: case 10: case 9: case 19: return 0;
    default: return 1; /* g = {G,P,A,T,S,N,H,Q,E,D,R,K} */
  }
}

static int class_pos3(int aa) {
  switch (aa) {
    case 0: return 0;                     /* A */
    case 4: return 1;                     /* C */
    case 13: case 18: case 17: return 2;  /* f = {F,Y,W} */
    case 7: return 3;                     /* G */
    case 9: case 19: return 4;            /* i = {I,V} */
    case 12: case 10: return 5;           /* m = {M,L} */
    case 2: case 8: return 6;             /* n = {N,H} */
    case 14: return 7;                    /* P */
    case 5: case 6: case 3: return 8;     /* q = {Q,E,D} */
    case 1: case 11: return 9;            /* r = {R,K} */
    default: return 10;                   /* t = {T,S}: codes 15, 16 */
  }
}

/* Class of residue aa at seed position pos (1..4); -1 for a stop or a code
 * outside the protein alphabet (such words are not indexed). */
int oracle_seed_class(int pos, int aa) {
  if (aa < 0 || aa >= NAA) return -1;
  if (pos == 1 || pos == 4) return aa;
  if (pos == 2) return class_pos2(aa);
  if (pos == 3) return class_pos3(aa);
  return -1;
}

/* Key of the W = 4 word starting at w[0], or -1 if a letter is not a residue. */
int32_t oracle_seed_key(const int8_t* w) {
  int c1 = oracle_seed_class(1, w[0]);
  int c2 = oracle_seed_class(2, w[1]);
  int c3 = oracle_seed_class(3, w[2]);
  int c4 = oracle_seed_class(4, w[3]);
  if (c1 < 0 || c2 < 0 || c3 < 0 || c4 < 0) return -1;
  return ((c1 * 2 + c2) * 11 + c3) * 20 + c4;
}

/* ------------------------------------------------------------------------
 * Stage 0, Section 3.3.1: index a bank.  Every overlapping word of length 4
 * inside one sequence (Section 2.3.1 splits a sequence into overlapping
 * words) is mapped to its subset-seed key; positions sharing a key are
 * linked.  The linked lists plus the look-up table of the paper are held as
 * one CSR array: key_off[k] .. key_off[k+1] are the positions of key k in
 * increasing order.  Positions are indices into the concatenated codes.
 * key_off must hold 8801 entries, pos must hold codes_len entries.
 * Returns the number of indexed positions.
 * ---------------------------------------------------------------------- */
int64_t oracle_index(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t* key_off, int32_t* pos) {
  int64_t* count = (int64_t*)calloc(NKEYS, sizeof(int64_t));
  for (int32_t s = 0; s < n_seqs; s++)
    for (int64_t p = seq_off[s]; p + 3 < seq_off[s + 1]; p++) {
      int32_t k = oracle_seed_key(codes + p);
      if (k >= 0) count[k]++;
    }
  key_off[0] = 0;
  for (int k = 0; k < NKEYS; k++) key_off[k + 1] = key_off[k] + count[k];
  /* fill in increasing position order: each list ends up sorted */
  memset(count, 0, NKEYS * sizeof(int64_t));
  for (int32_t s = 0; s < n_seqs; s++)
    for (int64_t p = seq_off[s]; p + 3 < seq_off[s + 1]; p++) {
      int32_t k = oracle_seed_key(codes + p);
      if (k >= 0) pos[key_off[k] + count[k]++] = (int32_t)p;
    }
  free(count);
  return key_off[NKEYS];
}

/* ------------------------------------------------------------------------
 * Parameters.  w: seed length (4).  nl / nr: neighbourhood residues left of
 * the seed start and right of the seed end (Section 3.3.2; the 48-residue
 * window of Annex 4 read as 22 + 4 + 22).  s1: ungapped threshold.
 * lg: residues per side of the small gapped extension.  band: half width of
 * the diagonal band.  gap_open / gap_extend: a gap of length k costs
 * gap_open + k * gap_extend.  s2: small gapped threshold.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t w, nl, nr, s1, lg, band, gap_open, gap_extend, s2;
  int32_t s0; /* Section 4.2's filter threshold; 0 = no filter */
} oracle_params;

/* ------------------------------------------------------------------------
 * Stage 2, Section 3.3.3 with the loop of Annex 4: ungapped score of the hit
 * whose seed starts at p1 in s1 and at p2 in s2.  The extension runs right
 * from the first seed letter over w + nr cells keeping a running sum and its
 * maximum (which starts at 0 and is raised only by a strictly larger sum);
 * the running sum is then set back to that maximum and the extension runs
 * left over nl cells.  The result is the final maximum, R + max(0, L).
 * Both parts are clipped at the ends of either sequence.
 * rlen: 1 + index of the first right cell reaching R (0 if R = 0).
 * llen: number of left cells up to the first one reaching the maximum
 *       (0 if the left part adds nothing).
 * ---------------------------------------------------------------------- */
int32_t oracle_ungapped_pair(const int8_t* s1, int64_t len1, int64_t p1, const int8_t* s2, int64_t len2, int64_t p2,
                             const oracle_params* prm, int32_t* rlen, int32_t* llen) {
  int64_t tr = prm->w + prm->nr;
  if (len1 - p1 < tr) tr = len1 - p1;
  if (len2 - p2 < tr) tr = len2 - p2;
  int64_t tl = prm->nl;
  if (p1 < tl) tl = p1;
  if (p2 < tl) tl = p2;

  int32_t sum = 0, best = 0, rl = 0, ll = 0;
  for (int64_t t = 0; t < tr; t++) {
    sum += B62[s1[p1 + t]][s2[p2 + t]];
    if (sum > best) {
      best = sum;
      rl = (int32_t)(t + 1);
    }
  }
  sum = best; /* the running sum restarts from the right maximum */
  for (int64_t t = 1; t <= tl; t++) {
    sum += B62[s1[p1 - t]][s2[p2 - t]];
    if (sum > best) {
      best = sum;
      ll = (int32_t)t;
    }
  }
  if (rlen) *rlen = rl;
  if (llen) *llen = ll;
  return best;
}

/* ------------------------------------------------------------------------
 * Section 4.2's filter: the raw score of two neighbourhoods is the sum of
 * the substitution scores of the residue pairs that score above zero,
 * taken here over the same window, clipped at the sequence ends the same
 * way, as the ungapped extension above (a reading: the paper's example uses
 * 12-residue subsequences; its filter runs on the neighbourhood blocks of
 * stage 2).  A pair goes on to the ungapped extension only if this score
 * reaches S0.
 * ---------------------------------------------------------------------- */
int32_t oracle_filter_pair(const int8_t* s1, int64_t len1, int64_t p1, const int8_t* s2, int64_t len2, int64_t p2,
                           const oracle_params* prm) {
  int64_t tr = prm->w + prm->nr;
  if (len1 - p1 < tr) tr = len1 - p1;
  if (len2 - p2 < tr) tr = len2 - p2;
  int64_t tl = prm->nl;
  if (p1 < tl) tl = p1;
  if (p2 < tl) tl = p2;
  int32_t f = 0;
  for (int64_t t = -tl; t < tr; t++) {
    int32_t sc = B62[s1[p1 + t]][s2[p2 + t]];
    if (sc > 0) f += sc;
  }
  return f;
}

/* ------------------------------------------------------------------------
 * Stage 3.1, Section 3.3.4: one side of the small gapped extension.
 * Dynamic programming (Gotoh's affine form) over A[1..la] x B[1..lb]
 * restricted to the diagonal band |i - j| <= band, anchored at (0, 0) with a
 * free end:
 *   H(0,0) = 0, cells outside the band or the grid are -infinity,
 *   E(i,j) = max(E(i,j-1) - ge, H(i,j-1) - go - ge)
 *   F(i,j) = max(F(i-1,j) - ge, H(i-1,j) - go - ge)
 *   H(i,j) = max(H(i-1,j-1) + s(A_i, B_j), E(i,j), F(i,j))
 * There is no clamp at zero.  The side score is the largest H over the band
 * (so at least H(0,0) = 0); *ei, *ej receive the first cell reaching it in
 * row-major order.  A and B are read through a stride so the same code
 * serves the right side (stride +1) and the left side (stride -1).
 * ---------------------------------------------------------------------- */
int32_t oracle_gapped_side(const int8_t* A, int64_t astride, int32_t la, const int8_t* B, int64_t bstride, int32_t lb,
                           int32_t band, int32_t go, int32_t ge, int32_t* ei, int32_t* ej) {
  int32_t w = lb + 1;
  int32_t* H = (int32_t*)malloc(sizeof(int32_t) * (size_t)(la + 1) * w);
  int32_t* E = (int32_t*)malloc(sizeof(int32_t) * (size_t)(la + 1) * w);
  int32_t* F = (int32_t*)malloc(sizeof(int32_t) * (size_t)(la + 1) * w);
  int32_t best = 0, bi = 0, bj = 0;
  for (int32_t i = 0; i <= la; i++) {
    for (int32_t j = 0; j <= lb; j++) {
      int32_t* h = &H[(size_t)i * w + j];
      int32_t* e = &E[(size_t)i * w + j];
      int32_t* f = &F[(size_t)i * w + j];
      int32_t d = i - j;
      if (d > band || -d > band) {
        *h = *e = *f = NEG_INF;
        continue;
      }
      if (i == 0 && j == 0) {
        *h = 0;
        *e = *f = NEG_INF;
        continue;
      }
      int32_t ev = NEG_INF, fv = NEG_INF, dv = NEG_INF;
      if (j > 0) {
        int32_t a = E[(size_t)i * w + j - 1] - ge;
        int32_t b = H[(size_t)i * w + j - 1] - go - ge;
        ev = a > b ? a : b;
      }
      if (i > 0) {
        int32_t a = F[(size_t)(i - 1) * w + j] - ge;
        int32_t b = H[(size_t)(i - 1) * w + j] - go - ge;
        fv = a > b ? a : b;
      }
      if (i > 0 && j > 0) {
        int32_t hd = H[(size_t)(i - 1) * w + j - 1];
        if (hd > NEG_INF / 2) dv = hd + B62[A[(i - 1) * astride]][B[(j - 1) * bstride]];
      }
      if (ev < NEG_INF / 2) ev = NEG_INF;
      if (fv < NEG_INF / 2) fv = NEG_INF;
      int32_t hv = dv;
      if (ev > hv) hv = ev;
      if (fv > hv) hv = fv;
      *h = hv;
      *e = ev;
      *f = fv;
      if (hv > best) {
        best = hv;
        bi = i;
        bj = j;
      }
    }
  }
  free(H);
  free(E);
  free(F);
  if (ei) *ei = bi;
  if (ej) *ej = bj;
  return best;
}

/* Small gapped score of a hit (Section 3.3.4 and the GPU description of
 * Section 5.2.2: one extension right of the seed start and one left of it).
 * Right: A = s1[p1 ..], B = s2[p2 ..], at most lg residues each, clipped at
 * the sequence ends.  Left: the residues before the anchor read backwards,
 * at most lg each, clipped at 0.  The score is right + left. */
int32_t oracle_small_gapped_pair(const int8_t* s1, int64_t len1, int64_t p1, const int8_t* s2, int64_t len2, int64_t p2,
                                 const oracle_params* prm, int32_t* r_i, int32_t* r_j, int32_t* l_i, int32_t* l_j) {
  int32_t la = (int32_t)((len1 - p1) < prm->lg ? (len1 - p1) : prm->lg);
  int32_t lb = (int32_t)((len2 - p2) < prm->lg ? (len2 - p2) : prm->lg);
  int32_t right = oracle_gapped_side(s1 + p1, 1, la, s2 + p2, 1, lb, prm->band, prm->gap_open, prm->gap_extend, r_i, r_j);
  la = (int32_t)(p1 < prm->lg ? p1 : prm->lg);
  lb = (int32_t)(p2 < prm->lg ? p2 : prm->lg);
  int32_t left = oracle_gapped_side(s1 + p1 - 1, -1, la, s2 + p2 - 1, -1, lb, prm->band, prm->gap_open,
                                    prm->gap_extend, l_i, l_j);
  return right + left;
}

/* ------------------------------------------------------------------------
 * Records.  Positions are local to their sequence.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t seq1, pos1, seq2, pos2;
  int16_t score;
  int8_t rlen, llen;
} oracle_hit;

typedef struct {
  int32_t seq1, pos1, seq2, pos2;
  int16_t score, ungapped;
  int16_t r_i, r_j, l_i, l_j;
} oracle_gapped;

static int cmp_hit(const void* a, const void* b) {
  const oracle_hit* x = (const oracle_hit*)a;
  const oracle_hit* y = (const oracle_hit*)b;
  if (x->seq1 != y->seq1) return x->seq1 < y->seq1 ? -1 : 1;
  if (x->pos1 != y->pos1) return x->pos1 < y->pos1 ? -1 : 1;
  if (x->seq2 != y->seq2) return x->seq2 < y->seq2 ? -1 : 1;
  if (x->pos2 != y->pos2) return x->pos2 < y->pos2 ? -1 : 1;
  return 0;
}

static int32_t seq_of(const int64_t* seq_off, int32_t n_seqs, int64_t p) {
  int32_t lo = 0, hi = n_seqs - 1; /* last s with seq_off[s] <= p */
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) / 2;
    if (seq_off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

typedef struct {
  const int8_t* codes;
  const int64_t* seq_off;
  int32_t n_seqs;
  const int64_t* key_off;
  const int32_t* pos;
} bank_view;

/* ------------------------------------------------------------------------
 * Stages 1 and 2 over a range of keys (Section 3.2's loop "for all possible
 * seeds"): for every key shared by the two banks, every pair of occurrences
 * is extended without gaps; pairs scoring at least s1 are kept.  Several
 * threads may share the work the way Section 5.1 shares seeds between
 * cores: a cursor under a mutex hands out the next piece of work, a key's
 * bank-1 occurrences a run at a time (runs of about 2^20 pairs, so that one
 * key with a very long list does not keep a single thread busy).  Each
 * thread keeps its own list; the lists are merged and sorted by (seq1, pos1,
 * seq2, pos2), so the result does not depend on the number of threads or on
 * how the work was cut.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t at;     /* index into the key range (or into key_list) */
  int64_t u_next; /* next bank-1 occurrence of that key; -1: not started */
} work_cursor;

typedef struct {
  const bank_view* b1;
  const bank_view* b2;
  const oracle_params* prm;
  const int32_t* key_list; /* NULL: keys are the cursor values themselves */
  int32_t key_hi;
  work_cursor* cursor;
  pthread_mutex_t* lock;
  oracle_hit* out;
  int64_t n, cap;
  int64_t pairs, filtered; /* pairs extended; of them, pairs through the filter */
} ungapped_job;

static void push_hit(ungapped_job* j, oracle_hit h) {
  if (j->n == j->cap) {
    j->cap = j->cap ? 2 * j->cap : 1024;
    j->out = (oracle_hit*)realloc(j->out, sizeof(oracle_hit) * (size_t)j->cap);
  }
  j->out[j->n++] = h;
}

/* The next piece of work: key *k, bank-1 occurrences [*u0, *u1).  Returns 0
 * when the range is exhausted.  Called with the lock held. */
static int next_work(ungapped_job* j, int32_t* k, int64_t* u0, int64_t* u1) {
  work_cursor* c = j->cursor;
  while (c->at < j->key_hi) {
    const int32_t key = j->key_list ? j->key_list[c->at] : c->at;
    const int64_t lo = j->b1->key_off[key], hi = j->b1->key_off[key + 1];
    const int64_t n2 = j->b2->key_off[key + 1] - j->b2->key_off[key];
    if (hi == lo || n2 == 0) {
      c->at++;
      c->u_next = -1;
      continue;
    }
    if (c->u_next < 0) c->u_next = lo;
    int64_t run = ((int64_t)1 << 20) / n2;
    if (run < 1) run = 1;
    *k = key;
    *u0 = c->u_next;
    *u1 = *u0 + run < hi ? *u0 + run : hi;
    c->u_next = *u1;
    if (*u1 == hi) {
      c->at++;
      c->u_next = -1;
    }
    return 1;
  }
  return 0;
}

static void* ungapped_worker(void* arg) {
  ungapped_job* j = (ungapped_job*)arg;
  const bank_view* b1 = j->b1;
  const bank_view* b2 = j->b2;
  for (;;) {
    int32_t k;
    int64_t ua, ub;
    pthread_mutex_lock(j->lock);
    const int more = next_work(j, &k, &ua, &ub);
    pthread_mutex_unlock(j->lock);
    if (!more) break;
    for (int64_t u = ua; u < ub; u++) {
      int64_t g1 = b1->pos[u];
      int32_t q1 = seq_of(b1->seq_off, b1->n_seqs, g1);
      int64_t o1 = b1->seq_off[q1];
      int64_t len1 = b1->seq_off[q1 + 1] - o1;
      for (int64_t v = b2->key_off[k]; v < b2->key_off[k + 1]; v++) {
        int64_t g2 = b2->pos[v];
        int32_t q2 = seq_of(b2->seq_off, b2->n_seqs, g2);
        int64_t o2 = b2->seq_off[q2];
        int64_t len2 = b2->seq_off[q2 + 1] - o2;
        j->pairs++;
        if (j->prm->s0 > 0 &&
            oracle_filter_pair(b1->codes + o1, len1, g1 - o1, b2->codes + o2, len2, g2 - o2, j->prm) < j->prm->s0)
          continue; /* Section 4.2: filtered out before the ungapped extension */
        j->filtered++;
        int32_t rl, ll;
        int32_t u_score = oracle_ungapped_pair(b1->codes + o1, len1, g1 - o1, b2->codes + o2, len2, g2 - o2, j->prm,
                                               &rl, &ll);
        if (u_score >= j->prm->s1) {
          oracle_hit h;
          h.seq1 = q1;
          h.pos1 = (int32_t)(g1 - o1);
          h.seq2 = q2;
          h.pos2 = (int32_t)(g2 - o2);
          h.score = (int16_t)u_score;
          h.rlen = (int8_t)rl;
          h.llen = (int8_t)ll;
          push_hit(j, h);
        }
      }
    }
  }
  return NULL;
}

/* Ungapped hits of all keys in [key_lo, key_hi), or, when key_list is not
 * NULL, of the keys key_list[key_lo .. key_hi).  *out is malloc'ed (free it
 * with oracle_free); *pairs receives the number of pairs extended.  Returns
 * the number of hits. */
int64_t oracle_ungapped(const int8_t* codes1, const int64_t* seq_off1, int32_t n1, const int64_t* key_off1,
                        const int32_t* pos1, const int8_t* codes2, const int64_t* seq_off2, int32_t n2,
                        const int64_t* key_off2, const int32_t* pos2, const oracle_params* prm, int32_t key_lo,
                        int32_t key_hi, const int32_t* key_list, int32_t n_threads, oracle_hit** out,
                        int64_t* pairs, int64_t* filtered) {
  bank_view b1 = {codes1, seq_off1, n1, key_off1, pos1};
  bank_view b2 = {codes2, seq_off2, n2, key_off2, pos2};
  if (n_threads < 1) n_threads = 1;
  work_cursor cursor = {key_lo, -1};
  pthread_mutex_t lock;
  pthread_mutex_init(&lock, NULL);
  ungapped_job* jobs = (ungapped_job*)calloc((size_t)n_threads, sizeof(ungapped_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int32_t t = 0; t < n_threads; t++) {
    jobs[t].b1 = &b1;
    jobs[t].b2 = &b2;
    jobs[t].prm = prm;
    jobs[t].key_list = key_list;
    jobs[t].key_hi = key_hi;
    jobs[t].cursor = &cursor;
    jobs[t].lock = &lock;
  }
  if (n_threads == 1) {
    ungapped_worker(&jobs[0]);
  } else {
    for (int32_t t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, ungapped_worker, &jobs[t]);
    for (int32_t t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
  }
  int64_t total = 0, npairs = 0, nfilt = 0;
  for (int32_t t = 0; t < n_threads; t++) {
    total += jobs[t].n;
    npairs += jobs[t].pairs;
    nfilt += jobs[t].filtered;
  }
  oracle_hit* all = (oracle_hit*)malloc(sizeof(oracle_hit) * (size_t)(total > 0 ? total : 1));
  int64_t at = 0;
  for (int32_t t = 0; t < n_threads; t++) {
    if (jobs[t].n) memcpy(all + at, jobs[t].out, sizeof(oracle_hit) * (size_t)jobs[t].n);
    at += jobs[t].n;
    free(jobs[t].out);
  }
  qsort(all, (size_t)total, sizeof(oracle_hit), cmp_hit);
  free(jobs);
  free(th);
  pthread_mutex_destroy(&lock);
  *out = all;
  if (pairs) *pairs = npairs;
  if (filtered) *filtered = nfilt;
  return total;
}

/* ------------------------------------------------------------------------
 * Stage 3.1 over a list of ungapped hits (Section 3.2: a hit scoring at
 * least S1 gets a small gapped extension, kept if it scores at least S2).
 * Output keeps the input order; *out is malloc'ed.  Returns the count.
 * With n_threads > 1 the hits are cut into that many consecutive ranges,
 * each extended by one thread into its own slots; the records are then
 * taken in input order, so the result does not depend on n_threads.
 * ---------------------------------------------------------------------- */
typedef struct {
  const int8_t *codes1, *codes2;
  const int64_t *seq_off1, *seq_off2;
  const oracle_params* prm;
  const oracle_hit* in;
  int64_t lo, hi;
  oracle_gapped* slot; /* one record per hit */
  char* keep;          /* G >= s2 per hit */
} gapped_job;

static void* gapped_worker(void* arg) {
  gapped_job* j = (gapped_job*)arg;
  for (int64_t u = j->lo; u < j->hi; u++) {
    const oracle_hit* h = &j->in[u];
    int64_t o1 = j->seq_off1[h->seq1], o2 = j->seq_off2[h->seq2];
    int64_t len1 = j->seq_off1[h->seq1 + 1] - o1, len2 = j->seq_off2[h->seq2 + 1] - o2;
    int32_t ri, rj, li, lj;
    int32_t g = oracle_small_gapped_pair(j->codes1 + o1, len1, h->pos1, j->codes2 + o2, len2, h->pos2, j->prm, &ri,
                                         &rj, &li, &lj);
    j->keep[u] = g >= j->prm->s2;
    oracle_gapped* r = &j->slot[u];
    r->seq1 = h->seq1;
    r->pos1 = h->pos1;
    r->seq2 = h->seq2;
    r->pos2 = h->pos2;
    r->score = (int16_t)g;
    r->ungapped = h->score;
    r->r_i = (int16_t)ri;
    r->r_j = (int16_t)rj;
    r->l_i = (int16_t)li;
    r->l_j = (int16_t)lj;
  }
  return NULL;
}

int64_t oracle_small_gapped(const int8_t* codes1, const int64_t* seq_off1, const int8_t* codes2,
                            const int64_t* seq_off2, const oracle_params* prm, const oracle_hit* in, int64_t n_in,
                            int32_t n_threads, oracle_gapped** out) {
  if (n_threads < 1) n_threads = 1;
  if (n_in < (int64_t)n_threads * 64) n_threads = 1;
  const size_t m = (size_t)(n_in > 0 ? n_in : 1);
  oracle_gapped* res = (oracle_gapped*)malloc(sizeof(oracle_gapped) * m);
  char* keep = (char*)malloc(m);
  gapped_job* jobs = (gapped_job*)calloc((size_t)n_threads, sizeof(gapped_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int32_t t = 0; t < n_threads; t++) {
    gapped_job* j = &jobs[t];
    j->codes1 = codes1;
    j->codes2 = codes2;
    j->seq_off1 = seq_off1;
    j->seq_off2 = seq_off2;
    j->prm = prm;
    j->in = in;
    j->lo = n_in * t / n_threads;
    j->hi = n_in * (t + 1) / n_threads;
    j->slot = res;
    j->keep = keep;
  }
  if (n_threads == 1) {
    gapped_worker(&jobs[0]);
  } else {
    for (int32_t t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, gapped_worker, &jobs[t]);
    for (int32_t t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
  }
  int64_t n = 0;
  for (int64_t u = 0; u < n_in; u++)
    if (keep[u]) res[n++] = res[u];
  free(keep);
  free(jobs);
  free(th);
  *out = res;
  return n;
}

void oracle_free(void* p) { free(p); }

/* ------------------------------------------------------------------------
 * Smith-Waterman local alignment with affine gaps (Gotoh 1982), textbook
 * form with the clamp at zero; a gap of length k costs go + k * ge.  Used
 * only as an upper bound on, and on tiny inputs the exact maximum of, the
 * small gapped scores.
 * ---------------------------------------------------------------------- */
int32_t oracle_smith_waterman(const int8_t* a, int32_t la, const int8_t* b, int32_t lb, int32_t go, int32_t ge) {
  int32_t w = lb + 1;
  int32_t* H = (int32_t*)calloc((size_t)(la + 1) * w, sizeof(int32_t));
  int32_t* E = (int32_t*)malloc(sizeof(int32_t) * (size_t)(la + 1) * w);
  int32_t* F = (int32_t*)malloc(sizeof(int32_t) * (size_t)(la + 1) * w);
  int32_t best = 0;
  for (int32_t i = 0; i <= la; i++)
    for (int32_t j = 0; j <= lb; j++) {
      size_t c = (size_t)i * w + j;
      E[c] = F[c] = NEG_INF;
      if (i == 0 || j == 0) continue;
      int32_t e1 = E[c - 1] - ge, e2 = H[c - 1] - go - ge;
      int32_t f1 = F[c - w] - ge, f2 = H[c - w] - go - ge;
      E[c] = e1 > e2 ? e1 : e2;
      F[c] = f1 > f2 ? f1 : f2;
      int32_t h = H[c - w - 1] + B62[a[i - 1]][b[j - 1]];
      if (E[c] > h) h = E[c];
      if (F[c] > h) h = F[c];
      if (h < 0) h = 0;
      H[c] = h;
      if (h > best) best = h;
    }
  free(H);
  free(E);
  free(F);
  return best;
}

/* ------------------------------------------------------------------------
 * Six-frame translation for TPLAST-N (Section 6 compares proteins with the
 * six translated frames of a nucleotide bank).  Standard genetic code
 * (NCBI translation table 1), written as the amino acid of every codon with
 * bases in the order T C A G for the first, second and third base.
 * Frames +1, +2, +3 read the contig from offsets 0, 1, 2; frames -1, -2, -3
 * read its reverse complement from offsets 0, 1, 2.  Only whole codons are
 * translated.  Sequences come out contig by contig, frames in the order
 * +1 +2 +3 -1 -2 -3; meta[2s] = contig, meta[2s+1] = frame (+-1..3).
 * Returns the number of amino acids written (aa must hold 2 * n_nt).
 * ---------------------------------------------------------------------- */
static const char GENETIC_CODE[65] = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG";

static int aa_code(char c) {
  static const char order[] = "ARNDCQEGHILKMFPSTWYV";
  if (c == '*') return STOP;
  for (int i = 0; i < 20; i++)
    if (order[i] == c) return i;
  return -1;
}

/* nucleotide code (A C G T = 0 1 2 3) to the T C A G index of the table */
static int tcag(int n) {
  switch (n) {
    case 3: return 0; /* T */
    case 1: return 1; /* C */
    case 0: return 2; /* A */
    default: return 3; /* G */
  }
}

int oracle_codon(int n1, int n2, int n3) { return aa_code(GENETIC_CODE[tcag(n1) * 16 + tcag(n2) * 4 + tcag(n3)]); }

int64_t oracle_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, int8_t* aa,
                          int64_t* seq_off, int32_t* meta) {
  int64_t at = 0;
  int32_t s = 0;
  seq_off[0] = 0;
  for (int32_t c = 0; c < n_contigs; c++) {
    const uint8_t* x = dna + contig_off[c];
    int64_t len = contig_off[c + 1] - contig_off[c];
    for (int32_t f = 0; f < 6; f++) {
      int64_t start = f % 3;
      for (int64_t p = start; p + 2 < len; p += 3) {
        int n1, n2, n3;
        if (f < 3) {
          n1 = x[p];
          n2 = x[p + 1];
          n3 = x[p + 2];
        } else { /* reverse complement: position q reads 3 - x[len - 1 - q] */
          n1 = 3 - x[len - 1 - p];
          n2 = 3 - x[len - 2 - p];
          n3 = 3 - x[len - 3 - p];
        }
        aa[at++] = (int8_t)oracle_codon(n1, n2, n3);
      }
      meta[2 * s] = c;
      meta[2 * s + 1] = f < 3 ? f + 1 : -(f - 2);
      seq_off[++s] = at;
    }
  }
  return at;
}
