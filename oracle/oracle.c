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
 *   xdrop_side / full_gapped .... Smith-Waterman bound and equality (no
 *                                 drop-off), hand-worked drop-off stops, the
 *                                 path rescored, redundancy worked by hand,
 *                                 input-order independence
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

/* ------------------------------------------------------------------------
 * Stage 3.2: full gapped extension (Section 3.3.4: a hit whose small gapped
 * extension reaches S2 gets "the standard dynamic programming procedure";
 * Section 2.3.3: a gapped extension stops once its score falls more than a
 * drop-off X below the best) and the trace-back of stage 4 (Section
 * 3.3.5) down to BLAST's tabular fields.  Readings:
 *  - anchor, sides, gap costs and the free end are those of stage 3.1: one
 *    extension right of the seed start (from its first residue pair) and one
 *    left of it, Gotoh with a gap of length k costing go + k * ge, no clamp
 *    at zero; but no band and no LG limit: a side runs to the sequence ends;
 *  - the drop-off is taken row by row: a cell whose H is more than X below
 *    T, the best H of all earlier rows (H(0,0) = 0 included), is dropped
 *    (H = E = F = minus infinity), and a side ends at its first row with no
 *    live cell;
 *  - the side's score is the best live H, its end the first cell holding it
 *    in row-major order;
 *  - the trace-back from the end cell prefers, in H, the diagonal, then E
 *    (gap in A: a B residue against nothing), then F (gap in B); in E or F it
 *    prefers the gap's opening over its extension when both give the value.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t lo, hi;    /* columns computed in this row (hi < lo: none) */
  int32_t *H, *E, *F; /* values of columns lo .. hi; dropped cells hold NEG_INF */
} xd_row;

static int32_t xd_get(const xd_row* r, const int32_t* v, int32_t j) {
  return (j < r->lo || j > r->hi) ? NEG_INF : v[j - r->lo];
}

/* One anchored side.  Rows i = 1..la take A_i = A[(i-1) * astride], columns
 * j = 1..lb take B_j = B[(j-1) * bstride].  Returns the side's score, its end
 * cell in (*ei, *ej), and the path from (0,0) to the end cell in ops[0 ..
 * *n_ops) from the anchor outwards: 'M' a residue pair, 'I' an A residue
 * against a gap, 'D' a B residue against a gap (ops holds la + lb). */
int32_t oracle_xdrop_side(const int8_t* A, int64_t astride, int32_t la, const int8_t* B, int64_t bstride, int32_t lb,
                          int32_t go, int32_t ge, int32_t X, int32_t* ei, int32_t* ej, char* ops, int32_t* n_ops) {
  const int32_t goe = go + ge;
  xd_row* rows = (xd_row*)calloc((size_t)la + 1, sizeof(xd_row));
  int32_t T = 0;       /* best H of the rows done so far */
  int32_t best = 0, bi = 0, bj = 0;
  int32_t last = -1;   /* last row with a live cell */
  for (int32_t i = 0; i <= la; i++) {
    const xd_row* up = i > 0 ? &rows[i - 1] : NULL;
    int32_t first = 0;
    if (up) {
      /* live cells of the row above bound where this row's can be */
      int32_t lo = INT32_MAX, hi = -1;
      for (int32_t j = up->lo; j <= up->hi; j++)
        if (up->H[j - up->lo] > NEG_INF) {
          if (j < lo) lo = j;
          hi = j;
        }
      if (hi < 0) break;
      first = lo;
    }
    /* columns first .. at most lb, stopping after the row above's live cells
     * end once a cell is dropped (nothing further right can be live) */
    int32_t cap = lb - first + 1;
    xd_row* r = &rows[i];
    r->lo = first;
    r->hi = first - 1;
    r->H = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    r->E = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    r->F = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    int32_t up_hi = -1;
    if (up)
      for (int32_t j = up->lo; j <= up->hi; j++)
        if (up->H[j - up->lo] > NEG_INF) up_hi = j;
    int32_t row_best = NEG_INF, row_bj = -1;
    for (int32_t j = first; j <= lb; j++) {
      int32_t h, e = NEG_INF, f = NEG_INF, d = NEG_INF;
      if (i == 0 && j == 0) {
        h = 0;
      } else {
        if (j > first) {
          const int32_t e1 = r->E[j - 1 - first], h1 = r->H[j - 1 - first];
          const int32_t a = e1 > NEG_INF ? e1 - ge : NEG_INF, b = h1 > NEG_INF ? h1 - goe : NEG_INF;
          e = a > b ? a : b;
        }
        if (up) {
          const int32_t f1 = xd_get(up, up->F, j), h1 = xd_get(up, up->H, j);
          const int32_t a = f1 > NEG_INF ? f1 - ge : NEG_INF, b = h1 > NEG_INF ? h1 - goe : NEG_INF;
          f = a > b ? a : b;
          const int32_t hd = j >= 1 ? xd_get(up, up->H, j - 1) : NEG_INF;
          if (hd > NEG_INF) d = hd + B62[A[(int64_t)(i - 1) * astride]][B[(int64_t)(j - 1) * bstride]];
        }
        h = d;
        if (e > h) h = e;
        if (f > h) h = f;
      }
      if (h < T - X) h = e = f = NEG_INF; /* dropped */
      r->H[j - first] = h;
      r->E[j - first] = e;
      r->F[j - first] = f;
      r->hi = j;
      if (h > row_best) {
        row_best = h;
        row_bj = j;
      }
      if (h == NEG_INF && j > up_hi) break;
    }
    if (row_best == NEG_INF) break; /* no live cell: the side ends */
    last = i;
    if (row_best > best) {
      best = row_best;
      bi = i;
      bj = row_bj;
    }
    if (row_best > T) T = row_best;
  }
  /* trace-back from (bi, bj) */
  int32_t n = 0, i = bi, j = bj;
  int state = 0; /* 0: H, 1: E, 2: F */
  while (i > 0 || j > 0) {
    const xd_row* r = &rows[i];
    if (state == 0) {
      const int32_t h = xd_get(r, r->H, j);
      const int32_t hd = (i >= 1 && j >= 1) ? xd_get(&rows[i - 1], rows[i - 1].H, j - 1) : NEG_INF;
      if (hd > NEG_INF && h == hd + B62[A[(int64_t)(i - 1) * astride]][B[(int64_t)(j - 1) * bstride]]) {
        ops[n++] = 'M';
        i--;
        j--;
      } else if (h == xd_get(r, r->E, j)) {
        state = 1;
      } else {
        state = 2;
      }
    } else if (state == 1) {
      const int32_t e = xd_get(r, r->E, j);
      const int32_t hl = xd_get(r, r->H, j - 1);
      ops[n++] = 'D';
      state = (hl > NEG_INF && e == hl - goe) ? 0 : 1;
      j--;
    } else {
      const int32_t f = xd_get(r, r->F, j);
      const int32_t hu = xd_get(&rows[i - 1], rows[i - 1].H, j);
      ops[n++] = 'I';
      state = (hu > NEG_INF && f == hu - goe) ? 0 : 2;
      i--;
    }
  }
  for (int32_t a = 0, b = n - 1; a < b; a++, b--) { /* anchor outwards */
    const char t = ops[a];
    ops[a] = ops[b];
    ops[b] = t;
  }
  *n_ops = n;
  *ei = bi;
  *ej = bj;
  (void)last;
  for (int32_t k = 0; k <= la; k++) {
    free(rows[k].H);
    free(rows[k].E);
    free(rows[k].F);
  }
  free(rows);
  return best;
}

typedef struct {
  int32_t seq1, seq2, pos1, pos2; /* the anchor: seed start of the hit it came from */
  int32_t score;                  /* right side + left side */
  int32_t q_start, q_end, s_start, s_end; /* aligned residues, 0-based, end exclusive */
  int32_t length, identities, mismatches, gap_opens;
} oracle_alignment;

typedef struct {
  int32_t diag, start, stop; /* an ungapped segment: pos1 - pos2, first and last pos1 */
} xd_segment;

/* Both sides of the anchor (p1, p2) of sequences s1 (len1) and s2 (len2):
 * score and tabular fields in *al, the alignment's ungapped segments
 * appended to *segs (growing *nseg / *capseg).  Gap runs are counted per
 * side (a run on each side of the anchor is two openings, as scored). */
int32_t oracle_full_gapped_pair(const int8_t* s1, int64_t len1, int64_t p1, const int8_t* s2, int64_t len2, int64_t p2,
                                int32_t go, int32_t ge, int32_t X, oracle_alignment* al, xd_segment** segs,
                                int32_t* nseg, int32_t* capseg) {
  const int32_t lar = (int32_t)(len1 - p1), lbr = (int32_t)(len2 - p2);
  const int32_t lal = (int32_t)p1, lbl = (int32_t)p2;
  char* opr = (char*)malloc((size_t)lar + lbr + 1);
  char* opl = (char*)malloc((size_t)lal + lbl + 1);
  int32_t ri, rj, li, lj, nr, nl;
  const int32_t right = oracle_xdrop_side(s1 + p1, 1, lar, s2 + p2, 1, lbr, go, ge, X, &ri, &rj, opr, &nr);
  const int32_t left = oracle_xdrop_side(s1 + p1 - 1, -1, lal, s2 + p2 - 1, -1, lbl, go, ge, X, &li, &lj, opl, &nl);
  al->pos1 = (int32_t)p1;
  al->pos2 = (int32_t)p2;
  al->score = right + left;
  al->q_start = (int32_t)p1 - li;
  al->q_end = (int32_t)p1 + ri;
  al->s_start = (int32_t)p2 - lj;
  al->s_end = (int32_t)p2 + rj;
  al->length = nl + nr;
  al->identities = al->mismatches = al->gap_opens = 0;
  /* columns in sequence order: the left path reversed, then the right path */
  int64_t x = p1 - li, y = p2 - lj;
  int32_t in_seg = 0;
  xd_segment cur = {0, 0, 0};
  for (int32_t c = 0; c < nl + nr; c++) {
    const int left_part = c < nl;
    const char op = left_part ? opl[nl - 1 - c] : opr[c - nl];
    const char prev = c == 0 || c == nl ? 0 : (left_part ? opl[nl - c] : opr[c - nl - 1]);
    if (op == 'M') {
      if (s1[x] == s2[y]) al->identities++;
      else al->mismatches++;
      if (in_seg && cur.diag == (int32_t)(x - y) && cur.stop == (int32_t)x - 1) {
        cur.stop = (int32_t)x;
      } else {
        if (in_seg) {
          if (*nseg == *capseg) {
            *capseg = *capseg ? 2 * *capseg : 16;
            *segs = (xd_segment*)realloc(*segs, sizeof(xd_segment) * (size_t)*capseg);
          }
          (*segs)[(*nseg)++] = cur;
        }
        cur.diag = (int32_t)(x - y);
        cur.start = cur.stop = (int32_t)x;
        in_seg = 1;
      }
      x++;
      y++;
    } else {
      if (op != prev) al->gap_opens++; /* a new run (runs do not cross the anchor) */
      if (op == 'I') x++;
      else y++;
    }
  }
  if (in_seg) {
    if (*nseg == *capseg) {
      *capseg = *capseg ? 2 * *capseg : 16;
      *segs = (xd_segment*)realloc(*segs, sizeof(xd_segment) * (size_t)*capseg);
    }
    (*segs)[(*nseg)++] = cur;
  }
  free(opr);
  free(opl);
  return al->score;
}

/* One anchor, for tests: the alignment and its ungapped segments as
 * (diagonal, start, stop) triples in seg_out[0 .. 3 * *n_seg) (at most cap
 * segments are copied; *n_seg is the full count). */
int32_t oracle_full_gapped_one(const int8_t* s1, int64_t len1, int64_t p1, const int8_t* s2, int64_t len2, int64_t p2,
                               int32_t go, int32_t ge, int32_t X, oracle_alignment* al, int32_t* seg_out, int32_t cap,
                               int32_t* n_seg) {
  xd_segment* segs = NULL;
  int32_t nseg = 0, capseg = 0;
  const int32_t sc = oracle_full_gapped_pair(s1, len1, p1, s2, len2, p2, go, ge, X, al, &segs, &nseg, &capseg);
  for (int32_t k = 0; k < nseg && k < cap; k++) {
    seg_out[3 * k] = segs[k].diag;
    seg_out[3 * k + 1] = segs[k].start;
    seg_out[3 * k + 2] = segs[k].stop;
  }
  *n_seg = nseg;
  free(segs);
  return sc;
}

/* ------------------------------------------------------------------------
 * Stage 3.2 over the stage-3.1 records, with the redundant-alignment lists
 * of Section 3.3.4: the ungapped segments (diagonal, start, stop) of every
 * gapped alignment computed are kept, and a hit lying on one of them (same
 * pair of sequences, same diagonal, pos1 between start and stop) is not
 * extended again.  The paper keeps the segments in k linked lists by
 * diagonal group; the result depends only on which segments exist, so this
 * statement keeps one plain list per pair of sequences.  Which hits are
 * skipped depends on the order they are taken in, which the paper leaves to
 * its streaming; here (a reading) the records of each pair are taken by
 * decreasing small gapped score, then increasing pos1, then pos2, so the
 * result does not depend on the input order.  Alignments scoring at least
 * s3 are returned, sorted by (seq1, pos1, seq2, pos2) of their anchor.
 * Pairs of sequences are independent: with n_threads > 1 they are shared
 * out in contiguous ranges.
 * ---------------------------------------------------------------------- */
typedef struct {
  const int8_t *codes1, *codes2;
  const int64_t *seq_off1, *seq_off2;
  int32_t go, ge, X;
  const oracle_gapped* in;
  const int64_t* order;     /* records grouped by pair, in processing order */
  const int64_t* group_at;  /* group g: order[group_at[g] .. group_at[g + 1]) */
  int64_t g_lo, g_hi;
  oracle_alignment* slot;   /* per record, in order[] positions */
  char* done;               /* 1: extended (not redundant) */
} full_job;

static const oracle_gapped* g_sort_in; /* qsort context (set before each sort, single-threaded) */

static int cmp_full_order(const void* a, const void* b) {
  const oracle_gapped* x = &g_sort_in[*(const int64_t*)a];
  const oracle_gapped* y = &g_sort_in[*(const int64_t*)b];
  if (x->seq1 != y->seq1) return x->seq1 < y->seq1 ? -1 : 1;
  if (x->seq2 != y->seq2) return x->seq2 < y->seq2 ? -1 : 1;
  if (x->score != y->score) return x->score > y->score ? -1 : 1;
  if (x->pos1 != y->pos1) return x->pos1 < y->pos1 ? -1 : 1;
  if (x->pos2 != y->pos2) return x->pos2 < y->pos2 ? -1 : 1;
  return 0;
}

static void* full_worker(void* arg) {
  full_job* j = (full_job*)arg;
  xd_segment* segs = NULL;
  int32_t nseg = 0, capseg = 0;
  for (int64_t g = j->g_lo; g < j->g_hi; g++) {
    nseg = 0;
    for (int64_t k = j->group_at[g]; k < j->group_at[g + 1]; k++) {
      const oracle_gapped* h = &j->in[j->order[k]];
      const int32_t d = h->pos1 - h->pos2;
      int redundant = 0;
      for (int32_t s = 0; s < nseg && !redundant; s++)
        redundant = segs[s].diag == d && segs[s].start <= h->pos1 && h->pos1 <= segs[s].stop;
      j->done[k] = 0;
      if (redundant) continue;
      const int64_t o1 = j->seq_off1[h->seq1], o2 = j->seq_off2[h->seq2];
      const int64_t len1 = j->seq_off1[h->seq1 + 1] - o1, len2 = j->seq_off2[h->seq2 + 1] - o2;
      oracle_alignment* al = &j->slot[k];
      oracle_full_gapped_pair(j->codes1 + o1, len1, h->pos1, j->codes2 + o2, len2, h->pos2, j->go, j->ge, j->X, al,
                              &segs, &nseg, &capseg);
      al->seq1 = h->seq1;
      al->seq2 = h->seq2;
      j->done[k] = 1;
    }
  }
  free(segs);
  return NULL;
}

static int cmp_alignment(const void* a, const void* b) {
  const oracle_alignment* x = (const oracle_alignment*)a;
  const oracle_alignment* y = (const oracle_alignment*)b;
  if (x->seq1 != y->seq1) return x->seq1 < y->seq1 ? -1 : 1;
  if (x->pos1 != y->pos1) return x->pos1 < y->pos1 ? -1 : 1;
  if (x->seq2 != y->seq2) return x->seq2 < y->seq2 ? -1 : 1;
  if (x->pos2 != y->pos2) return x->pos2 < y->pos2 ? -1 : 1;
  return 0;
}

/* Returns the number of alignments (malloc'ed in *out); *n_extended receives
 * how many records were extended (the rest were redundant). */
int64_t oracle_full_gapped(const int8_t* codes1, const int64_t* seq_off1, const int8_t* codes2,
                           const int64_t* seq_off2, int32_t go, int32_t ge, int32_t X, int32_t s3,
                           const oracle_gapped* in, int64_t n_in, int32_t n_threads, oracle_alignment** out,
                           int64_t* n_extended) {
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_in > 0 ? n_in : 1));
  for (int64_t k = 0; k < n_in; k++) order[k] = k;
  g_sort_in = in;
  qsort(order, (size_t)n_in, sizeof(int64_t), cmp_full_order);
  int64_t* group_at = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_in + 1));
  int64_t ng = 0;
  for (int64_t k = 0; k < n_in; k++)
    if (k == 0 || in[order[k]].seq1 != in[order[k - 1]].seq1 || in[order[k]].seq2 != in[order[k - 1]].seq2)
      group_at[ng++] = k;
  group_at[ng] = n_in;
  oracle_alignment* slot = (oracle_alignment*)calloc((size_t)(n_in > 0 ? n_in : 1), sizeof(oracle_alignment));
  char* done = (char*)calloc((size_t)(n_in > 0 ? n_in : 1), 1);
  if (n_threads < 1) n_threads = 1;
  if (ng < (int64_t)n_threads * 4) n_threads = 1;
  full_job* jobs = (full_job*)calloc((size_t)n_threads, sizeof(full_job));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int32_t t = 0; t < n_threads; t++) {
    full_job* j = &jobs[t];
    j->codes1 = codes1;
    j->codes2 = codes2;
    j->seq_off1 = seq_off1;
    j->seq_off2 = seq_off2;
    j->go = go;
    j->ge = ge;
    j->X = X;
    j->in = in;
    j->order = order;
    j->group_at = group_at;
    j->g_lo = ng * t / n_threads;
    j->g_hi = ng * (t + 1) / n_threads;
    j->slot = slot;
    j->done = done;
  }
  if (n_threads == 1) {
    full_worker(&jobs[0]);
  } else {
    for (int32_t t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, full_worker, &jobs[t]);
    for (int32_t t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
  }
  int64_t n = 0, ext = 0;
  for (int64_t k = 0; k < n_in; k++) {
    ext += done[k];
    if (done[k] && slot[k].score >= s3) slot[n++] = slot[k];
  }
  qsort(slot, (size_t)n, sizeof(oracle_alignment), cmp_alignment);
  free(order);
  free(group_at);
  free(done);
  free(jobs);
  free(th);
  *out = slot;
  if (n_extended) *n_extended = ext;
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
