/*
 * plast.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of
 * PLAST's bank-to-bank comparison (Nguyen & Lavenier, "Fine-grained
 * parallelization of similarity search between protein sequences", INRIA
 * RR-6513, 2008).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer to sequence data, offsets or records is a DEVICE pointer
 *   on the current CUDA device (for example a torch tensor's data_ptr()).
 *   Scalar outputs (n_out, n_aa_out, bank handles) are HOST pointers.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is queued on it; calls that return a count read that
 *   count back and therefore synchronise with the stream before returning.
 * - The caller owns every input and output buffer.  The library owns
 *   `plast_bank` objects (freed by plast_bank_free) and the scratch memory
 *   it allocates inside a call (stream-ordered, returned before the call
 *   returns).
 * - Return value: PLAST_OK (0) or a negative PLAST_E_* code; plast_strerror
 *   names it.  On PLAST_E_CAPACITY, *n_out holds the number of records the
 *   call needs and no record has been written.
 * - Residue codes (int8): 0..19 = A R N D C Q E G H I L K M F P S T W Y V,
 *   20 = stop '*' (translated banks).  Nucleotide codes (uint8): A C G T =
 *   0 1 2 3.  Any other code is PLAST_E_INVALID.
 * - Positions in records are 0-based and local to their sequence; seq1 /
 *   seq2 index the sequences of bank 1 / bank 2.
 * - Calls may come from several host threads at once, each on its own
 *   stream: a call's scratch and stage timers are its own, and a bank is
 *   only read once plast_index_bank has returned (it must outlive the calls
 *   that use it).  Exceptions: plast_small_gapped_noalloc (one static array
 *   per device) and the plast_set_* switches, which are process-wide and
 *   apply to the calls that start after them in every thread.
 */
#ifndef PLAST_H
#define PLAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLAST_OK 0
#define PLAST_E_INVALID (-1)  /* bad argument, code, offset or parameter */
#define PLAST_E_OOM (-2)      /* a device allocation failed */
#define PLAST_E_CAPACITY (-3) /* output buffer too small; *n_out = needed */
#define PLAST_E_CUDA (-4)     /* a CUDA runtime call or kernel failed */
#define PLAST_E_TIMEOUT (-5)  /* a bounded device-side wait expired (reserved: no
                                 kernel of this library waits on another CTA) */

#define PLAST_NKEYS 8800 /* subset-seed keys: 20 * 2 * 11 * 20 */
#define PLAST_MAX_STAGES 5 /* stage intervals reported by plast_stage_times */

/* Opaque, device-resident, library-owned indexed bank. */
typedef struct plast_bank plast_bank;

/*
 * Parameters (Section 3.2: thresholds S1, S2; Section 3.3.2 neighbourhoods;
 * Section 3.3.4 small gapped extension).
 *   w          seed length; must be 4 (the subset seed of Section 3.3.1)
 *   nl, nr     neighbourhood residues left of the seed start and right of
 *              the seed end; must be 22 and 22 (the 48-residue window of
 *              Annex 4, run as 26 cells right then 22 cells left)
 *   s1         ungapped threshold: a hit is kept if its score >= s1
 *   lg         residues per side of the small gapped extension; must be 64
 *   band       half width of the diagonal band; must be 8
 *   gap_open, gap_extend  a gap of length k costs gap_open + k*gap_extend
 *              (gap_open 0..1000, gap_extend 0..400: the small gapped
 *              extension keeps row i's values offset by i*gap_extend in
 *              int16)
 *   s2         small gapped threshold: kept if the score >= s2
 * Defaults (plast_default_params): 4, 22, 22, 38, 64, 8, 11, 1, 47.
 * Section 4.2's lossy filter threshold S0 is not a field: it is an argument
 * of plast_ungapped_ex, plast_search_ex and plast_plan_create, so that the
 * five calls of the boundary keep exactly this nine-field layout.
 */
typedef struct {
  int32_t w, nl, nr, s1, lg, band, gap_open, gap_extend, s2;
} plast_params;

/*
 * Filter threshold of Section 4.2 (the s0 argument of the _ex calls and of
 * plast_plan_create; 0 = no filter, at most 30000): a pair is kept by stage 2
 * only if, besides its ungapped score reaching s1, the sum of the positive
 * substitution scores over its window (clipped like the ungapped score)
 * reaches s0.  Lossy: it removes hits the unfiltered search keeps.
 * PLAST_FILTER_S0 is the value that lets about 2.5 % of random pairs
 * through, as the paper reports.
 */
#define PLAST_FILTER_S0 53

/*
 * Ungapped hit (stage 2).  score = R + max(0, L) as defined by Section
 * 3.3.3 and the loop of Annex 4; rlen = 1 + index of the first right cell
 * reaching R (0 if R = 0); llen = number of left cells up to the first one
 * reaching the final maximum (0 if the left part adds nothing).  20 bytes.
 */
typedef struct {
  int32_t seq1, pos1, seq2, pos2;
  int16_t score;
  int8_t rlen, llen;
} plast_hit;

/*
 * Small gapped extension (stage 3.1, Section 3.3.4): score = right side +
 * left side, ungapped = the stage-2 score of the same hit, (r_i, r_j) and
 * (l_i, l_j) = residues of bank 1 / bank 2 covered by the best cell of the
 * right and left side (first maximum in row-major order).  28 bytes.
 */
typedef struct {
  int32_t seq1, pos1, seq2, pos2;
  int16_t score, ungapped;
  int16_t r_i, r_j, l_i, l_j;
} plast_gapped;

/*
 * Full gapped alignment (stage 3.2, Section 3.3.4) with the tabular fields of
 * the trace-back (stage 4, Section 3.3.5; BLAST's -m 8 columns without the
 * E-value and bit score, which need statistics the paper does not give).
 * pos1 / pos2 are the seed start of the stage-3.1 record it was extended
 * from; [q_start, q_end) and [s_start, s_end) the aligned residues of the two
 * sequences (0-based, local); length = alignment columns; gap_opens counts
 * the gap runs of each side of the anchor (a run on each side of it is two).
 * 52 bytes.
 */
typedef struct {
  int32_t seq1, seq2, pos1, pos2;
  int32_t score;
  int32_t q_start, q_end, s_start, s_end;
  int32_t length, identities, mismatches, gap_opens;
} plast_alignment;

/* Stage-3.2 drop-off used when a caller has no other: 38, BLAST's
 * preliminary gapped drop-off of 15 bits at BLOSUM62 11/1's lambda 0.267. */
#define PLAST_XDROP 38

/* Fill *p with the default parameters listed above. */
void plast_default_params(plast_params* p);

/*
 * Six-frame translation of a nucleotide bank (Section 6, TPLAST-N: a protein
 * bank is compared with the six translated frames of a DNA bank).
 *   dna         [contig_off[n_contigs]] nucleotide codes 0..3 (device)
 *   contig_off  [n_contigs + 1] int64 offsets, contig_off[0] = 0 (device)
 *   aa_out      [aa_cap] residue codes 0..20 written here (device)
 *   seq_off_out [6 * n_contigs + 1] int64 offsets of the translated
 *               sequences (device)
 *   frame_meta_out [6 * n_contigs][2] int32 (contig, frame) per sequence,
 *               frame in +1 +2 +3 -1 -2 -3 (device)
 *   *n_aa_out   number of residues written (host)
 * Frames +f read the contig from offset f-1, frames -f its reverse
 * complement from offset f-1; only whole codons; standard genetic code
 * (NCBI table 1), stops as code 20.  Sequences are ordered contig by contig,
 * frames +1 +2 +3 -1 -2 -3.  Errors: PLAST_E_INVALID for a code > 3 or bad
 * offsets; PLAST_E_CAPACITY if aa_cap is too small (*n_aa_out = needed).
 */
int plast_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, int8_t* aa_out,
                     int64_t aa_cap, int64_t* seq_off_out, int32_t* frame_meta_out, int64_t* n_aa_out,
                     void* stream);

/*
 * Stage 0 (Section 3.3.1): index a bank by the subset seed.  Every word of
 * four residues inside one sequence (words holding a stop are skipped) is
 * mapped to its key; the positions of each key are kept in increasing
 * order, and the 48-residue neighbourhood of each position (Section 3.3.2)
 * is laid out next to it for stage 2.
 *   codes   [seq_off[n_seqs]] residue codes 0..20 (device)
 *   seq_off [n_seqs + 1] int64 offsets, seq_off[0] = 0, non-decreasing
 *           (device); total length < 2^31 - 2^26
 *   params  may be NULL (defaults)
 *   *out    receives the new bank (host)
 * The inputs are consumed before the call returns; the caller may free them
 * then.  The last step (laying out the neighbourhoods) may still be running
 * on `stream` when the call returns: every later call that takes the bank
 * waits for it, on whatever stream it is given, and plast_bank_free waits
 * too, so the caller may go on to host work (another bank, planning) while
 * it finishes.
 * Errors: PLAST_E_INVALID (code outside 0..20, bad offsets, n_seqs < 0,
 * unsupported params), PLAST_E_OOM, PLAST_E_CUDA.
 */
int plast_index_bank(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, const plast_params* params,
                     void* stream, plast_bank** out);

/* Release a bank and its device memory, after its construction has finished
 * (NULL is ignored). */
void plast_bank_free(plast_bank* bank);

/* Number of sequences / residues / indexed positions of a bank (host). */
int plast_bank_stats(const plast_bank* bank, int32_t* n_seqs, int64_t* n_residues, int64_t* n_positions);

/*
 * Copy a bank's index out: key_off [8801] int64 and pos [n] int32 global
 * residue indices (into the concatenated codes given to plast_index_bank),
 * increasing within each key (device pointers).  Section 3.3.1's look-up
 * table and linked lists in CSR form.  PLAST_E_CAPACITY if cap < n.
 */
int plast_bank_export_index(const plast_bank* bank, int64_t* key_off, int32_t* pos, int64_t cap, int64_t* n_out,
                            void* stream);

/*
 * Stages 1-2 (Sections 3.3.2-3.3.3, Annex 4): for every key present in both
 * banks, every pair of occurrences gets an ungapped extension; pairs scoring
 * >= params->s1 are written to out[0 .. *n_out) sorted by (seq1, pos1, seq2,
 * pos2).  out: [cap] plast_hit (device).
 * Errors: PLAST_E_INVALID, PLAST_E_CAPACITY (*n_out = needed), PLAST_E_OOM,
 * PLAST_E_CUDA, PLAST_E_TIMEOUT.
 */
int plast_ungapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params, plast_hit* out,
                   int64_t cap, int64_t* n_out, void* stream);

/*
 * plast_ungapped with two options the boundary call leaves out:
 *   s0     Section 4.2's filter threshold (0 = off; see PLAST_FILTER_S0)
 *   keys   host array of n_keys subset-seed keys (each 0..8799, duplicates
 *          ignored) to restrict the comparison to, or NULL for every key.
 *          Stages 1-3.1 are independent per key (Section 5.1 hands seeds to
 *          cores one at a time), so the hits of a key set are exactly the
 *          hits of the full call whose seed word has one of those keys.
 * plast_ungapped(b1, b2, p, out, cap, n, st) is
 * plast_ungapped_ex(b1, b2, p, 0, NULL, 0, out, cap, n, st).  Errors as
 * plast_ungapped, and PLAST_E_INVALID for s0 outside 0..30000, a key outside
 * 0..8799, or n_keys < 0.
 */
int plast_ungapped_ex(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                      const int32_t* keys, int32_t n_keys, plast_hit* out, int64_t cap, int64_t* n_out,
                      void* stream);

/*
 * Number of ungapped pairs (sum over keys of n1 * n2) the two banks give;
 * pure host arithmetic on the indexes, no device work.
 */
int64_t plast_pair_count(const plast_bank* b1, const plast_bank* b2);

/*
 * Stage 3.1 (Section 3.3.4, Section 5.2.2): small gapped extension of
 * n_in ungapped hits `in` (device; positions must be seed starts of the two
 * banks).  Hits scoring >= params->s2 are written to out in input order.
 * out: [cap] plast_gapped (device).  Errors as plast_ungapped.
 */
int plast_small_gapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params,
                       const plast_hit* in, int64_t n_in, plast_gapped* out, int64_t cap, int64_t* n_out,
                       void* stream);

/*
 * Stages 1-3.1 in one call (Section 3.2's loop without stages 3.2 and 4):
 * ungapped extension of every pair, small gapped extension of the hits
 * scoring >= s1, and the records scoring >= s2 written to out sorted by
 * (seq1, pos1, seq2, pos2).  Errors as plast_ungapped (and PLAST_E_CAPACITY
 * when a call has 2^32 or more stage-2 hits).
 */
int plast_search(const plast_bank* b1, const plast_bank* b2, const plast_params* params, plast_gapped* out,
                 int64_t cap, int64_t* n_out, void* stream);

/*
 * plast_search with the options of plast_ungapped_ex (s0, keys / n_keys,
 * NULL keys = every key) and one more output: *n_ungapped_out (host, may be
 * NULL) receives the number of stage-2 hits (those through the S0 filter
 * when s0 > 0).  plast_search(b1, b2, p, out, cap, n, st) is
 * plast_search_ex(b1, b2, p, 0, NULL, 0, out, cap, n, NULL, st).
 */
int plast_search_ex(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                    const int32_t* keys, int32_t n_keys, plast_gapped* out, int64_t cap, int64_t* n_out,
                    int64_t* n_ungapped_out, void* stream);

/*
 * Stage 3.2 and the trace-back (Sections 3.3.4 and 3.3.5) of n_in stage-3.1
 * records `in` (device, any order; as plast_search returns them): each is
 * extended with gaps in both directions from its seed start, without band or
 * length limit, the extension of a side stopping at the first row whose
 * cells all lie more than `xdrop` below the best of the rows before
 * (PLAST_XDROP if unsure).  Section 3.3.4's redundancy lists: for each pair of
 * sequences the records are taken by decreasing small gapped score, then by
 * position, and a record whose seed start lies on a gap-free segment
 * (diagonal, first and last residue) of an alignment already computed for
 * that pair is not extended.  Alignments scoring >= s3 are written to out
 * sorted by (seq1, pos1, seq2, pos2); *n_extended_out (host, may be NULL)
 * receives how many records were extended.  Gap costs come from params.
 * Errors as plast_small_gapped, plus PLAST_E_INVALID for xdrop outside
 * 0..30000 or banks of more than 2^24 sequences each, and PLAST_E_CAPACITY
 * (with *n_out = 0) when an extension outgrows the kernel's working space: a
 * row of more than 1024 computed columns, more than about half a million cells
 * for one side, or more than 8192 gap-free segments for one pair of
 * sequences.
 */
int plast_full_gapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t xdrop,
                      int32_t s3, const plast_gapped* in, int64_t n_in, plast_alignment* out, int64_t cap,
                      int64_t* n_out, int64_t* n_extended_out, void* stream);

/*
 * The dynamic-programming cells that the last plast_full_gapped call made on
 * this host thread computed: every cell of every row of every extended side,
 * the dropped ones included (the unit of stage 3.2's throughput).  0 before
 * the first call and after a call that failed.
 */
int64_t plast_full_gapped_cells(void);

/*
 * plast_small_gapped without device allocation.  The paper has no
 * counterpart to this call; it exists for callers that cannot let a library
 * allocate device memory: a framework that reserved the GPU's memory for its
 * own allocator, or a latency-bound loop that must not meet an allocation's
 * implicit synchronisation or an out-of-memory failure mid-request.
 * Same arguments, results and errors as plast_small_gapped, except:
 *  - n_in must be at most PLAST_NOALLOC_MAX_HITS (otherwise PLAST_E_INVALID);
 *  - the working buffers live in one static device array of
 *    PLAST_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that
 *    loads the library until the process exits; no cudaMalloc or cudaFree
 *    is called;
 *  - every call on a device uses that same array, which keeps the previous
 *    call's contents: calls whose work overlaps on the GPU (other streams,
 *    other threads) race and must be serialised by the caller;
 *  - the first call on a device performs one-time set-up (it looks up the
 *    array's device address and loads the score tables into constant
 *    memory); make that first call before any stream capture.  That set-up
 *    is kept for the life of the process: after cudaDeviceReset (or
 *    anything else that replaces the device's primary context) the address
 *    is stale, so do not call into the library again in that process.
 */
#define PLAST_NOALLOC_MAX_HITS 65536
#define PLAST_NOALLOC_SCRATCH_BYTES (2 * 1024 * 1024 + 8192)
int plast_small_gapped_noalloc(const plast_bank* b1, const plast_bank* b2, const plast_params* params,
                               const plast_hit* in, int64_t n_in, plast_gapped* out, int64_t cap,
                               int64_t* n_out, void* stream);

/*
 * Planned search for repeated comparisons of the same two banks (a resident
 * bank against a fixed query set, a benchmark loop).  plast_plan_create
 * allocates every buffer the search needs for at most max_hits stage-2 hits
 * and uploads the stage-2 work list; `records` (device, caller-owned,
 * max_records entries) receives the stage-3.1 records of every run.  The
 * banks and `records` must outlive the plan.  plast_plan_run then queues the
 * whole chain of stages 1-3.1 on `stream` with no allocation and no host
 * synchronisation (the kernels pass the survivor count in device memory), so
 * it can be captured in a CUDA graph; plast_plan_capture does that capture
 * on a non-default `stream` and keeps the instantiated graph in the plan,
 * and plast_plan_launch replays it.  plast_plan_result synchronises `stream`
 * and returns the record count of the last run (records in canonical order,
 * as plast_search) and its stage-2 hit count (those through the S0 filter
 * when s0 > 0, s0 as in plast_search_ex; max_hits bounds the count before
 * it); PLAST_E_CAPACITY if either
 * limit was exceeded (*n_records then holds the hit or record count that did
 * not fit, and the records are an incomplete subset).  PLAST_E_INVALID at
 * creation unless max_records >= 1 and 1 <= max_hits < 2^32.  Runs of one
 * plan must not overlap on the device.
 */
typedef struct plast_plan plast_plan;
int plast_plan_create(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                      int64_t max_hits, plast_gapped* records, int64_t max_records, void* stream,
                      plast_plan** out);
int plast_plan_run(plast_plan* plan, void* stream);
int plast_plan_capture(plast_plan* plan, void* stream);
int plast_plan_launch(plast_plan* plan, void* stream);
int plast_plan_result(const plast_plan* plan, int64_t* n_records, int64_t* n_hits, void* stream);
void plast_plan_free(plast_plan* plan);

/*
 * Fault injection for the failure paths (tests): from now on every device
 * allocation the library makes larger than `bytes` fails as if the device
 * were out of memory, and the call reports PLAST_E_OOM with everything it had
 * allocated freed; 0 removes the limit.  PLAST_E_INVALID if bytes < 0.
 * Applies to later calls in this process.
 */
int plast_set_alloc_limit(int64_t bytes);

/*
 * Scheduling of stage 2.  0 (default): one persistent launch, CTAs pull
 * profile tiles from a device work queue, largest first.  1: the plain
 * form, one launch per key.  Applies to later calls in this process.
 */
int plast_set_schedule(int mode);

/*
 * Stage-2 tile shapes.  The work of a key is cut into tiles of consecutive
 * bank-1 occurrences: wide tiles of 128 rows, whose profile serves 4 bank-2
 * windows per warp, and narrow tiles of 16, 8, 4 or 2 rows, one bank-2
 * window per lane, for short lists (a small query bank against a large one,
 * the end of a long list).  After the full wide tiles of a key, the library
 * covers the remainder either with one wide tile or with narrow tiles (16
 * rows while 16 or more remain, or 8 if those cost less per row, the last
 * rows by the cheapest cover with 16, 8, 4 and 2 rows), from a cost model: a
 * tile of shape S costs
 * S_slot x (rows of S) x ceil(n2 / P_S) x P_S + S_tile SM-nanoseconds, n2 the
 * key's bank-2 occurrences, P_S the bank-2 windows a CTA scores per pass
 * (128 wide, 512 narrow).  plast_autotune measures the constants on the
 * current device (random banks, the stage-2 kernel timed with every tile of
 * one shape, against a long and a short bank 2; about a second), installs
 * them and copies them to *out (may be NULL).  It also picks the wide kernel
 * variant by timing each: how many cells of the wide profile are held as
 * int16 (no sign extension, twice the shared-memory traffic), then how many
 * passes ahead a warp fetches its next bank-2 windows (the staging depth).
 * plast_get_tile_costs / plast_set_tile_costs read and install costs and
 * variant (for a cached calibration; PLAST_E_INVALID unless the slot costs
 * are positive, the tile costs non-negative, wide_int16_cells one of the
 * variants and wide_stage_depth 0, 1 or 2).  plast_set_tile_shape forces the shape of every tile (1 wide;
 * 2, 3, 4, 5 narrow of 8, 4, 2, 16 rows; 0, the default, by cost).  Shapes change
 * the schedule, never the results.  Settings are process-wide and apply to
 * later calls.
 */
typedef struct plast_tile_costs {
  double wide_slot, wide_tile;       /* 128 rows */
  double narrow_slot, narrow_tile;   /* 8 rows */
  double narrow4_slot, narrow4_tile; /* 4 rows */
  double narrow2_slot, narrow2_tile; /* 2 rows */
  int32_t wide_int16_cells; /* kernel variant: cells of the wide profile held as int16 (0, 12, 14 or 16) */
  int32_t wide_stage_depth; /* kernel variant: bank-2 windows fetched 1 or 2 passes ahead (0 = 1) */
  double narrow16_slot, narrow16_tile; /* 16 rows */
} plast_tile_costs;
int plast_autotune(void* stream, plast_tile_costs* out);
int plast_get_tile_costs(plast_tile_costs* out);
int plast_set_tile_costs(const plast_tile_costs* costs);
int plast_set_tile_shape(int mode);
/*
 * The stage-2 work list the library would run for two banks with the given
 * CSR key offsets (host arrays of PLAST_NKEYS + 1 entries each, as
 * plast_bank_export_index returns) on a GPU of n_sms SMs (0: no splitting of
 * long lists): host-only, no device needed.  Fills tiles[6 * t ..] with (key,
 * first bank-1 CSR index, rows, shape: 0 wide, 1, 2, 3, 4 narrow of 8, 4, 2,
 * 16 rows, first and end offset of its bank-2 windows in the key's list) in
 * launch order for t < *n_tiles; PLAST_E_CAPACITY if more than `cap` tiles
 * (then *n_tiles = needed), PLAST_E_INVALID on decreasing offsets.
 */
int plast_stage2_tiles(const int64_t* key_off1, const int64_t* key_off2, int32_t n_sms, int32_t* tiles, int64_t cap,
                       int64_t* n_tiles);

/*
 * Instrumentation (no effect on results).
 * plast_set_timing(1) makes later plast_ungapped / plast_small_gapped /
 * plast_search calls (of every thread) record CUDA events on their stream
 * at the stage boundaries; plast_stage_times then fills ms[0 .. n) with the
 * device time of the intervals of the calling thread's last such call (-1
 * where not recorded):
 *   ms[0] work list upload   ms[1] stage-2 kernel   ms[2] survivor count read
 *   (and, for plast_ungapped, the survivor sort)   ms[3] stage-3.1 kernel
 *   ms[4] threshold scan, record sort (plast_search) and write-out.
 * plast_kernel_launches returns how many kernels the library has launched in
 * this process so far.
 */
int plast_set_timing(int on);
int plast_stage_times(double* ms, int n);
long long plast_kernel_launches(void);

/* Static name of a PLAST_OK / PLAST_E_* return code. */
const char* plast_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PLAST_H */
