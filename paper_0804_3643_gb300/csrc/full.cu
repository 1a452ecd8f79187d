// full.cu -- stage 3.2 (Section 3.3.4: the full gapped extension of the hits
// whose small gapped extension reaches S2, with the list of ungapped segments
// that keeps a hit lying on an alignment already found from being extended
// again) and the trace-back of stage 4 (Section 3.3.5) down to BLAST's
// tabular fields, on sm_103a.
//
// Work split.  The records of one pair of sequences depend on one another
// through the segment list, so one warp takes all the records of a pair, in
// the processing order (decreasing small gapped score, then pos1, then
// pos2); pairs are independent, and a warp takes the next one from a shared
// counter when it is done with the last.
//
// One side of one record is an anchored dynamic programme without a band,
// cut by the drop-off X row by row: a cell whose H is more than X below T,
// the best H of the rows before it, is dropped (H = F = minus infinity).  The
// warp computes a row 32 columns at a time, one column per lane, from the
// first live column of the row above:
//   F  = max(F_up - ge, H_up - go - ge)        (shared memory: the row above)
//   D  = H_diag + s(A_i, B_j)
//   DF = max(D, F)
//   E  = max over k < j in the row of DF(k) - go - (j - k) ge
//      = (exclusive prefix maximum of DF(k) + k ge) - go - j ge   (warp scan)
//   H  = max(DF, E)
// E here is not reset at dropped cells; a value that reaches a cell through a
// dropped one is already below T - X there, so it neither keeps a cell alive
// nor equals the H of a live cell, and the scores, end cells and paths are
// those of the row-by-row statement.  A row stops at the first chunk past
// the row above's live cells whose last cell is dropped (beyond them only E
// feeds a cell, and it only falls).
//
// Each live cell leaves its H (int16, relative to its row's drop-off line)
// in the warp's arena (global memory), a dead one a dead marker.  After the
// side's last row, the warp walks back from the end cell (first maximum in
// row-major order) to the anchor, 32 steps at a time, taking at each cell
// the source the recurrences give in the order of preference diagonal, E,
// F, and opening a gap in preference to extending one of equal value, all
// from the stored H values of the cell's row and the row above (an E is
// recomputed along its row when the diagonal does not give the cell's H);
// it counts the
// alignment's columns, identities and gap runs and emits its gap-free
// segments (diagonal pos1 - pos2, first and last pos1).
//
// Limits (reported as PLAST_E_CAPACITY by the call): a row of more than
// FG_W computed columns, more than FG_ARENA bytes of H values and row table
// for one side, more than FG_SEGS segments for one pair of sequences (and,
// as a guard that no path the recurrences give can trip, a walk leaving
// the grid).
#include <stdint.h>

#include "common.cuh"
#include "full.cuh"

namespace plast {

constexpr int FG_WARPS = 4;  // warps per CTA
constexpr int32_t FG_NEG = -(1 << 28);
constexpr int FG_SMEM = FG_WARPS * (FG_W + 4) * 4;  // per warp: one row of (H, F) int16 slots

// The row above is kept in shared memory as int16 values relative to its
// drop-off line thr = T - X, one 32-bit slot per column (H in the low half,
// F in the high half): a live cell's H lies in [thr, thr + X + 11] (no cell
// rises more than one diagonal step, at most 11, above the best of the
// earlier rows), and a dead cell is stored as -30000 in both halves.
// Decoded, such a value lies 30,000 below the line and everything computed
// from it (adding a score, subtracting gap costs) stays below the line of
// this row and of every later one, so it can neither keep a cell alive nor
// equal the H of a live cell: the scores, end cells and paths are those of
// minus infinity, with no test per use.  A live cell's F needs no clamp: it
// comes from a dead slot (so it lies within go + ge + 11 of -30000) or from
// a live H above (within go + ge of the line), so it stays in int16.  Slots
// 0 and 1 of the row buffer hold the dead value too, and a column past the
// row above's last stored one reads as dead (one compare on the slot), so
// the row below reads out-of-range columns with no other test.
constexpr int FG_DEAD16 = -30000;
constexpr uint32_t FG_DEAD = 0x8AD08AD0u;  // FG_DEAD16 in both halves
constexpr int FG_SLOTS = FG_W + 4;  // the row buffer: two dead slots before the row, two spare

// One side of one anchor.  Row i takes A_i = A[DIR (i - 1)], column j takes
// B_j = B[DIR (j - 1)]; la / lb residues.  Returns the side's score, its end
// cell and its computed cells; the H values and the row table (origin,
// offset, line, stored columns per row) are in `arena`.  *err gets FG_ERR_*
// bits on a capacity overflow.
//
// A row is computed 64 columns at a time, two adjacent columns j0 = cs + 2l
// and j0 + 1 per lane, from an even origin o at or left of the row's first
// column c0 (the column left of c0 that the rounding may add comes out
// dead and is not counted), so that a row of the random extensions (about
// 40 columns) takes one pass and one scan.  Column j is kept in slot
// j - o + 2 (slots 0 and 1 hold the dead value), so the two slots a lane
// reads and writes are one aligned 8-byte word; the E scan runs over the
// lanes' pairwise maxima.  Values are computed relative to the line of the
// row above (the stored int16 decode with no add), the live test and the
// stored values relative to the row's own line.  Each lane keeps, over the
// row's chunks, its first and last live column and its best key (H - line)
// << 11 | (2047 - (j - o)) of a live cell; three warp reductions at the
// row's end give the live window, the row maximum and its first column.
struct SideOut {
  int32_t score, ei, ej;
  int64_t cells;  // computed cells, every row
};

template <int DIR>
__device__ SideOut side_dp(const int8_t* A, int la, const int8_t* B, int lb, int go, int ge, int X, const int8_t* tab,
                           uint32_t* Sbuf, uint8_t* arena, int* err, int lane) {
  const int goe = go + ge;
  int32_t* rowtab = reinterpret_cast<int32_t*>(arena);  // (origin, offset, line, stored columns) per row
  int16_t* hval = reinterpret_cast<int16_t*>(arena);     // H of the stored columns, from the offset
  const int64_t tab_bytes = (int64_t)16 * (la + 1);
  SideOut out = {0, 0, 0, 0};
  if (tab_bytes > FG_ARENA) {
    if (lane == 0) atomicOr(err, FG_ERR_ARENA);
    return out;
  }
  int off = (int)(tab_bytes / 2);  // in int16 units, even
  // a side whose rows all fit whole, even at their widest (la + 1 rows of at
  // most lb + 2 stored columns), needs no capacity test at all
  const bool side_fits = lb + 4 <= FG_W && off + (int64_t)(la + 1) * (lb + 2) < FG_ARENA / 2;
  int32_t T = 0, best = 0, bi = 0, bj = 0;
  int32_t cells = 0;  // computed cells (at most the arena's columns)
  int plo = 0, phi = 0, po = 0, pw2 = 2;  // the row above: live columns, origin, first slot after it
  int32_t pthr = 0;                       // the row above's drop-off line
  int ai = 0;                             // A_i of the row (row 0: none)
  __syncwarp();  // (row 0 has no row above: pw2 = 2 makes it an empty one)
  for (int i = 0; i <= la; i++) {
    const int c0 = i == 0 ? 0 : plo;
    const int o = c0 & ~1;                 // the row's origin (even)
    const int lim = i == 0 ? 0 : phi + 1;  // the last column a cell of the row above can feed
    // the row is written over the row above in the same buffer: a chunk
    // reads the row above before it stores (its scan's shuffles come
    // between), the row's origin is never left of the row above's, so a
    // chunk overwrites only columns left of what later chunks read, but for
    // the row-above column just left of the next chunk, which lane 31 of
    // this chunk hands on
    uint32_t* Sp = Sbuf;
    uint32_t carry_sm = 0;  // the row above's slot of column cs - 1 (chunks after the first)
    const int32_t thr = T - X;
    const int32_t trel = thr - pthr;  // the row's line relative to the row above's
    const int8_t* trow = tab + ai * NCODE;
    ai = i < la ? A[DIR * i] : 0;  // the next row's residue, loaded a row ahead
    int32_t carryP = FG_NEG;
    int32_t lkey = -1, llo = 0x7fffffff, lhi = -1;  // this lane's best key, first and last live column
    bool overflow = false;
    // a row that fits whole needs no test per chunk
    const bool fits = side_fits || (lb - o + 4 <= FG_W && off + (lb - o) + 1 < FG_ARENA / 2);
    int cs = o;  // (o <= c0 <= lb: the row has at least one chunk)
    for (;; cs += 64) {
      // capacity of the chunk's last column (the same test for every lane)
      const int wl = min(cs + 63, lb) - o;
      if (!fits && (wl + 4 > FG_W || off + wl + 1 >= FG_ARENA / 2)) {
        overflow = true;
        break;
      }
      // (a column left of c0 reads only dead cells of the row above and dead
      // E terms: it comes out dead, and its prefix term lies below every
      // live one to its right; a column past lb feeds only columns past lb)
      const int j0 = cs + 2 * lane, j1 = j0 + 1;
      const bool in0 = j0 <= lb, in1 = j1 <= lb;
      // row above: columns j0 and j0 + 1 at slots kp, kp + 1 (kp = j0 - po +
      // 2, even; the load stays inside the buffer), column j0 - 1 from the
      // lane to the left (lane 0: from lane 31 of the chunk before, and in a
      // row's first chunk column o - 1, left of the row above's first live
      // column, dead)
      const int kp = j0 - po + 2;
      // (the slots from pw2 on may hold this row's own earlier chunks: a
      // column there is past the row above and takes the dead value)
      uint2 sv = *reinterpret_cast<const uint2*>(Sp + min(kp, pw2));
      if (kp >= pw2) sv = make_uint2(FG_DEAD, FG_DEAD);
      uint32_t sm = __shfl_up_sync(0xffffffffu, sv.y, 1);
      if (lane == 0) sm = cs > o ? carry_sm : FG_DEAD;
      const int32_t hd0 = (int32_t)(int16_t)(sm & 0xffffu);
      const int32_t hu0 = (int32_t)(int16_t)(sv.x & 0xffffu), fu0 = (int32_t)sv.x >> 16;
      const int32_t hu1 = (int32_t)(int16_t)(sv.y & 0xffffu), fu1 = (int32_t)sv.y >> 16;
      // (j = 0 and columns past the sequence end read the sentinel padding)
      const int32_t D0 = hd0 + trow[B[DIR * (j0 - 1)]], D1 = hu0 + trow[B[DIR * j0]];
      const int32_t F0 = max(fu0 - ge, hu0 - goe), F1 = max(fu1 - ge, hu1 - goe);
      int32_t DF0 = max(D0, F0);
      const int32_t DF1 = max(D1, F1);
      if (i == 0 && j0 == 0) DF0 = 0;  // the anchor (row 0's row above is empty, its line 0)
      // E from the exclusive prefix maximum of DF(k) + k ge over the row (a
      // lane below the shuffle distance gets its own value back)
      const int32_t P0 = DF0 + j0 * ge, P1 = DF1 + j1 * ge;
      int32_t incl = max(P0, P1);
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) incl = max(incl, __shfl_up_sync(0xffffffffu, incl, d));
      int32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
      ex = lane == 0 ? carryP : max(ex, carryP);
      const int32_t E0 = ex - go - j0 * ge, E1 = max(ex, P0) - go - j1 * ge;
      const int32_t H0 = max(DF0, E0), H1 = max(DF1, E1);
      const bool live0 = in0 && H0 >= trel, live1 = in1 && H1 >= trel;
      const int32_t r0 = H0 - trel, r1 = H1 - trel;  // against the row's line
      if (in0 || in1) {
        const int w = j0 - o;  // even
        const uint32_t v0 = live0 ? __byte_perm((uint32_t)r0, (uint32_t)(F0 - trel), 0x5410u) : FG_DEAD;
        const uint32_t v1 = live1 ? __byte_perm((uint32_t)r1, (uint32_t)(F1 - trel), 0x5410u) : FG_DEAD;
        *reinterpret_cast<uint2*>(Sp + w + 2) = make_uint2(v0, v1);
        *reinterpret_cast<uint32_t*>(hval + off + w) = __byte_perm(v0, v1, 0x5410u);  // the two H halves
      }
      // (the key as r * 2048 + code: r >= 0 and code < 2048 for a live cell;
      // a multiply-add leaves the ALU pipe, the bound, to the maxima)
      const int kc = 2047 - (j0 - o);
      lkey = max(lkey, max(live0 ? r0 * 2048 + kc : -1, live1 ? r1 * 2048 + (kc - 1) : -1));
      llo = min(llo, live0 ? j0 : live1 ? j1 : 0x7fffffff);
      lhi = max(lhi, live1 ? j1 : live0 ? j0 : -1);
      // past the sequence end, or past the row above's reach with the
      // chunk's last cell dropped: the row ends
      if (cs + 64 > lb || (cs + 63 >= lim && !(__ballot_sync(0xffffffffu, live1) >> 31))) break;
      // what the next chunk takes from this one's lane 31
      carryP = max(carryP, __shfl_sync(0xffffffffu, incl, 31));
      carry_sm = __shfl_sync(0xffffffffu, sv.y, 31);
    }
    if (overflow) {
      if (lane == 0) atomicOr(err, FG_ERR_WIDTH);
      return out;
    }
    const int cend = min(cs + 64, lb + 1);  // past the row's last computed column
    const int cw = (cend - o + 1) & ~1;     // stored columns, even
    cells += cend - c0;
    const int32_t key = __reduce_max_sync(0xffffffffu, lkey);
    if (key < 0) break;  // no live cell: the side ends
    const int32_t rmax = (key >> 11) + thr;
    const int rarg = o + 2047 - (key & 2047);
    plo = __reduce_min_sync(0xffffffffu, llo);
    phi = __reduce_max_sync(0xffffffffu, lhi);
    if (lane == 0) *reinterpret_cast<int4*>(rowtab + 4 * i) = make_int4(o, off, thr, cw);
    off += cw;
    if (rmax > best) {
      best = rmax;
      bi = i;
      bj = rarg;
    }
    T = max(T, rmax);
    po = o;
    pw2 = cw + 2;
    pthr = thr;
    __syncwarp();
  }
  out.score = best;
  out.ei = bi;
  out.ej = bj;
  out.cells = cells;
  return out;
}

// The path of a side from its end cell back to the anchor.  Columns (cell
// (i, j) holds residues x = x0 + dx * (i - 1), y = y0 + dy * (j - 1) of the
// padded banks) are counted into *st; gap-free runs are appended to segs
// (pos1 coordinates are local: x - xoff), except the run that reaches the
// anchor, returned in *anchor_run (valid when its length is > 0).
struct PathStats {
  int32_t length, identities, mismatches, gap_opens;
};
struct Run {
  int32_t diag, start, stop, len;
};

// A row's table entry (origin, offset, line, stored columns) as one 16-byte
// load, and H(i, j) of that row from it (FG_NEG where the cell is dead or was
// not computed).
__device__ __forceinline__ int4 row_entry(const uint8_t* arena, int i) {
  return *reinterpret_cast<const int4*>(arena + 16 * (int64_t)i);
}
__device__ __forceinline__ int32_t entry_h(const int16_t* hval, const int4& t, int j) {
  const int k = j - t.x;
  if (k < 0 || k >= t.w) return FG_NEG;
  const int v = hval[t.y + k];
  return v == FG_DEAD16 ? FG_NEG : v + t.z;
}

// The whole warp walks the path of a side from its end cell (ei, ej), whose
// H is `score`, back to the anchor; every lane keeps the same state.  Row i
// takes A_i = pad1[x1 + dir (i - 1)], column j B_j = pad2[y1 + dir (j - 1)].
// At a cell in state H the diagonal is taken when H = H(i - 1, j - 1) +
// s(A_i, B_j) with the diagonal cell live, else E when H equals the row's E
// there (max over the live cells k < j of the row of H(i, k) - go - (j - k)
// ge, the value the extension's prefix maximum gives: a term through a
// dropped cell lies below the line), else F; a gap opens at the first cell
// back where its value equals the live neighbour's H - go - ge.  The steps
// are tested 32 at a time, lane t taking the t-th: a run of diagonal steps
// ends at the first lane whose test fails (one ballot), a gap at the first
// lane whose cell closes it, and the E of a cell is one warp maximum of
// H(i, k) + k ge over the row.  Columns are counted into *st; gap-free runs
// are appended to segs by lane 0 (pos1 coordinates are local: x - xoff),
// except the run that reaches the anchor, returned in *anchor_run (valid
// when its length is > 0).  A path that would leave the grid (the
// recurrences never lead there) stops with FG_ERR_PATH.
__device__ void walk_side(const uint8_t* arena, int ei, int ej, int32_t score, const int8_t* pad1,
                          const int8_t* pad2, int64_t x1, int64_t y1, int dir, int64_t xoff, int64_t yoff, int go,
                          int ge, const int8_t* tab, PathStats* st, int32_t* segs, int* nseg, int* err,
                          Run* anchor_run, int lane) {
  const unsigned FULL = 0xffffffffu;
  const int goe = go + ge;
  const int16_t* hval = reinterpret_cast<const int16_t*>(arena);
  int i = ei, j = ej, state = 0, prev_gap = 0;
  int32_t v = score;  // the value of the current state at (i, j)
  Run cur = {0, 0, 0, 0};
  auto flush = [&](bool at_anchor) {
    if (cur.len == 0) return;
    if (at_anchor) {
      *anchor_run = cur;
    } else if (*nseg < FG_SEGS) {
      if (lane == 0) {
        segs[3 * *nseg] = cur.diag;
        segs[3 * *nseg + 1] = cur.start;
        segs[3 * *nseg + 2] = cur.stop;
      }
      (*nseg)++;
    } else if (lane == 0) {
      atomicOr(err, FG_ERR_SEGS);
    }
    cur.len = 0;
  };
  while (i > 0 || j > 0) {
    if (i < 0 || j < 0) {
      if (lane == 0) atomicOr(err, FG_ERR_PATH);
      break;
    }
    if (state == 0) {
      // diagonal steps: lane t tests cell (i - t, j - t) against (i - t - 1,
      // j - t - 1), the value there being the H the step before it reaches
      const int it = i - lane, jt = j - lane;
      const bool on = it > 0 && jt > 0;
      int32_t hd = FG_NEG, sc = 0;
      bool ident = false;
      if (on) {
        const int64_t x = x1 + (int64_t)dir * (it - 1), y = y1 + (int64_t)dir * (jt - 1);
        const int ra = pad1[x], rb = pad2[y];
        hd = entry_h(hval, row_entry(arena, it - 1), jt - 1);
        sc = tab[ra * NCODE + rb];
        ident = ra == rb;
      }
      int32_t vt = __shfl_up_sync(FULL, hd, 1);
      if (lane == 0) vt = v;
      const unsigned okm = __ballot_sync(FULL, on && hd > FG_NEG && vt == hd + sc);
      const unsigned idm = __ballot_sync(FULL, ident);
      const int k = okm == FULL ? 32 : __ffs(~okm) - 1;  // leading diagonal steps
      if (k > 0) {
        const unsigned km = k == 32 ? FULL : (1u << k) - 1u;
        const int nid = __popc(idm & km);
        st->identities += nid;
        st->mismatches += k - nid;
        st->length += k;
        // residue pairs (A_{i-t}, B_{j-t}), t < k: one diagonal, pos1 px0 - dir t
        const int32_t px0 = (int32_t)(x1 + (int64_t)dir * (i - 1) - xoff);
        const int32_t py0 = (int32_t)(y1 + (int64_t)dir * (j - 1) - yoff);
        const int32_t pxl = px0 - dir * (k - 1);
        const int32_t lo = min(px0, pxl), hi = max(px0, pxl);
        if (cur.len > 0 && cur.diag == px0 - py0) {
          cur.start = min(cur.start, lo);
          cur.stop = max(cur.stop, hi);
          cur.len += k;
        } else {
          flush(false);
          cur.diag = px0 - py0;
          cur.start = lo;
          cur.stop = hi;
          cur.len = k;
        }
        prev_gap = 0;
        v = __shfl_sync(FULL, hd, k - 1);
        i -= k;
        j -= k;
      }
      if (k < 32 && (i > 0 || j > 0)) {
        // E of the cell from its row: max over the live k < j of
        // H(i, k) - goe - (j - 1 - k) ge
        const int4 tc = row_entry(arena, i);
        int32_t m = FG_NEG;
        for (int c = tc.x + lane; c < j; c += 32) {
          const int32_t h = entry_h(hval, tc, c);
          if (h > FG_NEG) m = max(m, h + c * ge);
        }
        m = __reduce_max_sync(FULL, m);
        const int32_t e = m > FG_NEG ? m - goe - (j - 1) * ge : FG_NEG;
        state = v == e ? 1 : 2;
        // (row 0 has no F and column 0 no E: the recurrences never lead
        // there; the walk stays on the grid regardless)
        if (i == 0) state = 1;
        else if (j == 0) state = 2;
      }
    } else {
      flush(false);  // a gap ends the current run
      if (prev_gap != state) st->gap_opens++;
      prev_gap = state;
      // a run is a stretch of equal gap columns, whatever the path's
      // opening decisions (with a free opening a run may open twice).  Lane
      // t tests the t-th step: its value v + t ge against the live
      // neighbour's H - goe (left for E, above for F)
      int32_t hn = FG_NEG;
      if (state == 1) {  // gap in A: B_j against nothing
        if (j - lane - 1 >= 0) hn = entry_h(hval, row_entry(arena, i), j - lane - 1);
      } else {           // gap in B: A_i against nothing
        if (i - lane - 1 >= 0) hn = entry_h(hval, row_entry(arena, i - lane - 1), j);
      }
      const unsigned cm = __ballot_sync(FULL, hn > FG_NEG && v + lane * ge == hn - goe);
      const int n = cm ? __ffs(cm) : 32;  // steps taken
      st->length += n;
      if (cm) {
        v = __shfl_sync(FULL, hn, n - 1);
        state = 0;
      } else {
        v += 32 * ge;
      }
      if (prev_gap == 1) j -= n;
      else i -= n;
    }
  }
  flush(true);
}

__global__ void __launch_bounds__(FG_WARPS * 32, 6) k_full_gapped(FullArgs a) {
  __shared__ int8_t tab[NCODE * NCODE];
  extern __shared__ __align__(16) int16_t fsm[];
  for (int t = threadIdx.x; t < NCODE * NCODE; t += blockDim.x) tab[t] = c_score[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* Sbuf = reinterpret_cast<uint32_t*>(fsm) + warp * FG_SLOTS;
  if (lane == 0) Sbuf[0] = Sbuf[1] = FG_DEAD;  // never written
  const int64_t gw = (int64_t)blockIdx.x * FG_WARPS + warp;
  uint8_t* arena = a.arena + gw * FG_ARENA;
  int32_t* segs = a.segs + gw * 3 * FG_SEGS;
  const int64_t ng = *a.ng_dev;
  for (;;) {
    // the next pair of sequences from a shared counter: pairs differ widely
    // in work, and a fixed share per warp left a fifth of the warps' time
    // idle at the end
    unsigned gn = 0;
    if (lane == 0) gn = atomicAdd(a.next, 1u);
    const int64_t g = (int64_t)__shfl_sync(0xffffffffu, gn, 0);
    if (g >= ng) break;
    int nseg = 0;
    for (int64_t k = a.gstart[g]; k < a.gstart[g + 1]; k++) {
      const uint32_t rec = a.proc[k];
      const plast_gapped r = a.in[rec];
      // the redundancy check: the anchor on a segment of this pair's list
      const int32_t dg = r.pos1 - r.pos2;
      bool on = false;
      for (int s = lane; s < nseg; s += 32)
        on |= segs[3 * s] == dg && segs[3 * s + 1] <= r.pos1 && r.pos1 <= segs[3 * s + 2];
      if (__any_sync(0xffffffffu, on)) {
        if (lane == 0) a.done[rec] = 0;
        continue;
      }
      const int64_t s1 = a.pad_off1[r.seq1], s2 = a.pad_off2[r.seq2];
      const int len1 = (int)(a.pad_off1[r.seq1 + 1] - s1 - GAP), len2 = (int)(a.pad_off2[r.seq2 + 1] - s2 - GAP);
      const int64_t x0 = s1 + r.pos1, y0 = s2 + r.pos2;  // padded anchor
      // right side: rows A_1.. = pad1[x0 ..], columns pad2[y0 ..]
      const SideOut R = side_dp<1>(a.pad1 + x0, len1 - r.pos1, a.pad2 + y0, len2 - r.pos2, a.go, a.ge, a.xdrop, tab,
                                   Sbuf, arena, a.err, lane);
      __syncwarp();
      PathStats st = {0, 0, 0, 0};
      Run rr = {0, 0, 0, 0}, lr = {0, 0, 0, 0};
      walk_side(arena, R.ei, R.ej, R.score, a.pad1, a.pad2, x0, y0, 1, s1, s2, a.go, a.ge, tab, &st, segs, &nseg,
                a.err, &rr, lane);
      __syncwarp();
      // left side: rows A_1.. = pad1[x0 - 1 ..] backwards
      const SideOut L = side_dp<-1>(a.pad1 + x0 - 1, r.pos1, a.pad2 + y0 - 1, r.pos2, a.go, a.ge, a.xdrop, tab, Sbuf,
                                    arena, a.err, lane);
      __syncwarp();
      walk_side(arena, L.ei, L.ej, L.score, a.pad1, a.pad2, x0 - 1, y0 - 1, -1, s1, s2, a.go, a.ge, tab, &st, segs,
                &nseg, a.err, &lr, lane);
      if (lane == 0) {
        // the runs that reach the anchor from both sides are one segment
        if (rr.len > 0 || lr.len > 0) {
          Run m = rr.len > 0 ? rr : lr;
          if (rr.len > 0 && lr.len > 0) m.start = lr.start;
          if (nseg < FG_SEGS) {
            segs[3 * nseg] = m.diag;
            segs[3 * nseg + 1] = m.start;
            segs[3 * nseg + 2] = m.stop;
            nseg++;
          } else {
            atomicOr(a.err, FG_ERR_SEGS);
          }
        }
        plast_alignment al;
        al.seq1 = r.seq1;
        al.seq2 = r.seq2;
        al.pos1 = r.pos1;
        al.pos2 = r.pos2;
        al.score = R.score + L.score;
        al.q_start = r.pos1 - L.ei;
        al.q_end = r.pos1 + R.ei;
        al.s_start = r.pos2 - L.ej;
        al.s_end = r.pos2 + R.ej;
        al.length = st.length;
        al.identities = st.identities;
        al.mismatches = st.mismatches;
        al.gap_opens = st.gap_opens;
        a.res[rec] = al;
        a.done[rec] = 1;
        atomicAdd(a.cells, (unsigned long long)(R.cells + L.cells));
      }
      nseg = __shfl_sync(0xffffffffu, nseg, 0);
      __syncwarp();
    }
  }
}

cudaError_t launch_full_gapped(const FullArgs& a, int64_t warps, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_full_gapped, cudaFuncAttributeMaxDynamicSharedMemorySize, FG_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (warps <= 0) return cudaSuccess;
  note_launch();
  k_full_gapped<<<(unsigned)(warps / FG_WARPS), FG_WARPS * 32, FG_SMEM, st>>>(a);
  return cudaGetLastError();
}

int64_t full_gapped_warps(int n_sms) { return (int64_t)n_sms * 6 * FG_WARPS; }

// ---------------------------------------------------------------------------
// Ordering and output
// ---------------------------------------------------------------------------
// Canonical key (padded pos1 << sh | padded pos2) of each record, with the
// record's fields checked against the banks (bad |= 1 otherwise).
__global__ void k_full_canon(const plast_gapped* in, int64_t n, const int64_t* po1, int32_t n1, const int64_t* po2,
                             int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n; h += (int64_t)gridDim.x * blockDim.x) {
    const plast_gapped r = in[h];
    bool ok = r.seq1 >= 0 && r.seq1 < n1 && r.seq2 >= 0 && r.seq2 < n2;
    int64_t p1 = 0, p2 = 0;
    if (ok) {
      const int64_t l1 = po1[r.seq1 + 1] - po1[r.seq1] - GAP, l2 = po2[r.seq2 + 1] - po2[r.seq2] - GAP;
      ok = r.pos1 >= 0 && r.pos1 < l1 && r.pos2 >= 0 && r.pos2 < l2;
      p1 = po1[r.seq1] + r.pos1;
      p2 = po2[r.seq2] + r.pos2;
    }
    if (!ok) {
      atomicOr(bad, 1);
      p1 = p2 = 0;
    }
    key[h] = ((uint64_t)p1 << sh) | (uint64_t)p2;
    val[h] = (uint32_t)h;
  }
}

// Processing key of the records in canonical order: (seq1, seq2, 32767 -
// small gapped score); sorted stably after the canonical sort, ties keep
// (pos1, pos2) order.
__global__ void k_full_proc(const plast_gapped* in, const uint32_t* canon, int64_t n, int b2, uint64_t* key,
                            uint32_t* val) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = canon[c];
    const plast_gapped r = in[h];
    key[c] = ((((uint64_t)(uint32_t)r.seq1 << b2) | (uint64_t)(uint32_t)r.seq2) << 16) |
             (uint64_t)(uint16_t)(32767 - (int32_t)r.score);
    val[c] = h;
  }
}

// flag[k] = 1 where a new pair of sequences starts in processing order
__global__ void k_full_group_flags(const plast_gapped* in, const uint32_t* proc, int64_t n, int32_t* flag) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const plast_gapped r = in[proc[k]];
    bool head = k == 0;
    if (!head) {
      const plast_gapped q = in[proc[k - 1]];
      head = q.seq1 != r.seq1 || q.seq2 != r.seq2;
    }
    flag[k] = head;
  }
}

__global__ void k_full_group_starts(const int32_t* flag, const int64_t* at, int64_t n, const int64_t* ng,
                                    int64_t* gstart) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (flag[k]) gstart[at[k]] = k;
  if (blockIdx.x == 0 && threadIdx.x == 0) gstart[*ng] = n;
}

// keep[c] = the record at canonical position c was extended and scores >= s3
__global__ void k_full_keep(const uint32_t* canon, int64_t n, const int32_t* done, const plast_alignment* res,
                            int32_t s3, int32_t* keep) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = canon[c];
    keep[c] = done[h] && res[h].score >= s3;
  }
}

__global__ void k_full_write(const uint32_t* canon, int64_t n, const int32_t* keep, const int64_t* at,
                             const plast_alignment* res, plast_alignment* out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (keep[c]) out[at[c]] = res[canon[c]];
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b > 0 ? b : 1);
}

cudaError_t launch_full_canon(const plast_gapped* in, int64_t n, const int64_t* po1, int32_t n1, const int64_t* po2,
                              int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  k_full_canon<<<grid_for(n), 256, 0, st>>>(in, n, po1, n1, po2, n2, sh, key, val, bad);
  return cudaGetLastError();
}

cudaError_t launch_full_proc(const plast_gapped* in, const uint32_t* canon, int64_t n, int b2, uint64_t* key,
                             uint32_t* val, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  k_full_proc<<<grid_for(n), 256, 0, st>>>(in, canon, n, b2, key, val);
  return cudaGetLastError();
}

cudaError_t launch_full_groups(const plast_gapped* in, const uint32_t* proc, int64_t n, int32_t* flag,
                               const int64_t* at, const int64_t* ng, int64_t* gstart, int phase, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  if (phase == 0) k_full_group_flags<<<grid_for(n), 256, 0, st>>>(in, proc, n, flag);
  else k_full_group_starts<<<grid_for(n), 256, 0, st>>>(flag, at, n, ng, gstart);
  return cudaGetLastError();
}

cudaError_t launch_full_keep(const uint32_t* canon, int64_t n, const int32_t* done, const plast_alignment* res,
                             int32_t s3, int32_t* keep, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  k_full_keep<<<grid_for(n), 256, 0, st>>>(canon, n, done, res, s3, keep);
  return cudaGetLastError();
}

cudaError_t launch_full_write(const uint32_t* canon, int64_t n, const int32_t* keep, const int64_t* at,
                              const plast_alignment* res, plast_alignment* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  k_full_write<<<grid_for(n), 256, 0, st>>>(canon, n, keep, at, res, out);
  return cudaGetLastError();
}

}  // namespace plast
