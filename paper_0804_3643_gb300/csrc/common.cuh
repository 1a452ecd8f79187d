// common.cuh -- constants, tables and helpers of the CUDA library.
//
// Residue codes: 0..19 = A R N D C Q E G H I L K M F P S T W Y V, 20 = stop,
// 21 = SENTINEL, the code of the padding the library writes between the
// sequences of a bank.  Every score involving the sentinel is SENT_SCORE,
// which is negative: an extension that runs past a sequence end meets only
// sentinels from there on, so its running sum falls strictly and its
// maximum is the one of the clipped window (Section 3.3.3 / Annex 4 with
// windows clipped at the sequence ends).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/plast.h"

namespace plast {

constexpr int NAA = 20;
constexpr int STOP = 20;
constexpr int SENTINEL = 21;
constexpr int NCODE = 22;          // residues, stop, sentinel
constexpr int SENT_SCORE = -32;    // score of any pair involving the sentinel
constexpr int NKEYS = PLAST_NKEYS; // 20 * 2 * 11 * 20

// Neighbourhood window of stage 2 (Annex 4: 48 = 3 x 16 cells; read as
// 26 cells right of the seed start, seed included, then 22 cells left).
constexpr int WIN = 48;
constexpr int RIGHT = 26;
constexpr int LEFT = 22;

// Small gapped extension (Section 3.3.4): LG residues per side, band |i-j|<=BAND.
constexpr int LG = 64;
constexpr int BAND = 8;
constexpr int BW = 2 * BAND + 1;

// Sentinel gap written before, between and after the sequences of a bank.
// It must cover the farthest read past a sequence end: 26 cells of the
// ungapped window, and LG + BAND = 72 residues of the gapped band.
constexpr int GAP = 80;

// Launch geometry of the stage-2 kernel.
constexpr int UNG_T1 = 128;        // bank-1 rows per wide profile tile
constexpr int UNG_NT1 = 8;         // bank-1 rows per narrow profile tile
constexpr int UNG_THREADS = 768;   // 24 warps (85 registers a thread), one CTA per SM

// BLOSUM62, upper triangle by rows, order A R N D C Q E G H I L K M F P S T W Y V
// (Henikoff & Henikoff 1992).  Expanded to a 22 x 22 table with the stop row
// (-4 against residues, +1 against stop) and the sentinel row by
// build_score_table().
static const char* const B62_UPPER[20] = {
    "4 -1 -2 -2 0 -1 -1 0 -2 -1 -1 -1 -1 -2 -1 1 0 -3 -2 0",
    "5 0 -2 -3 1 0 -2 0 -3 -2 2 -1 -3 -2 -1 -1 -3 -2 -3",
    "6 1 -3 0 0 0 1 -3 -3 0 -2 -3 -2 1 0 -4 -2 -3",
    "6 -3 0 2 -1 -1 -3 -4 -1 -3 -3 -1 0 -1 -4 -3 -3",
    "9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1",
    "5 2 -2 0 -3 -2 1 0 -3 -1 0 -1 -2 -1 -2",
    "5 -2 0 -3 -3 1 -2 -3 -1 0 -1 -3 -2 -2",
    "6 -2 -4 -4 -2 -3 -3 -2 0 -2 -2 -3 -3",
    "8 -3 -3 -1 -2 -1 -2 -1 -2 -2 2 -3",
    "4 2 -3 1 0 -3 -2 -1 -3 -1 3",
    "4 -2 2 0 -3 -2 -1 -2 -1 1",
    "5 -1 -3 -1 0 -1 -3 -2 -2",
    "5 0 -2 -1 -1 -1 -1 1",
    "6 -4 -2 -2 1 3 -1",
    "7 -1 -1 -4 -3 -2",
    "4 1 -3 -2 -2",
    "5 -2 -2 0",
    "11 2 -3",
    "7 -1",
    "4",
};

// Subset seed of Section 3.3.1 as class member lists.  Positions 1 and 4 are
// the identity on the 20 residues (the printed list misses I: its own class).
// Position 3 prints f = {F,Y,E}; read as {F,Y,W}.
static const char* const SEED_POS2[2] = {"CFYWMLIV", "GPATSNHQEDRK"};
static const char* const SEED_POS3[11] = {"A", "C", "FYW", "G", "IV", "ML", "NH", "P", "QED", "RK", "TS"};
static const char* const ALPHABET = "ARNDCQEGHILKMFPSTWYV";

struct Tables {
  int8_t score[NCODE * NCODE];  // score[a * NCODE + b]
  int8_t cls2[NAA];
  int8_t cls3[NAA];
};

// Host: expand the transcriptions above into the tables the kernels use.
void build_tables(Tables* t);

// Device copies (constant memory), filled once per device by upload_tables().
extern __constant__ int8_t c_score[NCODE * NCODE];
extern __constant__ int8_t c_cls2[NAA];
extern __constant__ int8_t c_cls3[NAA];

// One byte from shared memory at a 32-bit shared address plus a constant
// offset.  Issued as its own load so the byte goes through the load/store
// unit rather than being carved out of a wider load on the integer ALU.
template <int OFF>
__device__ __forceinline__ uint32_t lds_u8(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1+%2];" : "=r"(v) : "r"(saddr), "n"(OFF));
  return v;
}

// Host: the parameter checks every entry point applies (NULL = defaults).
// The kernels fix w, the window, LG and the band; gap costs are bounded so
// that the small gapped extension's offset rows stay inside int16.
inline bool params_ok(const plast_params* p) {
  if (!p) return true;
  return p->w == 4 && p->nl == LEFT && p->nr == RIGHT - 4 && p->lg == LG && p->band == BAND && p->gap_open >= 0 &&
         p->gap_extend >= 0 && p->gap_open <= 1000 && p->gap_extend <= 400 && p->s1 >= -30000 &&
         p->s1 <= 30000 && p->s2 >= -30000 && p->s2 <= 30000;
}

// Host: the parameters a call runs with (the defaults for NULL).
inline plast_params resolve(const plast_params* p) {
  plast_params d;
  plast_default_params(&d);
  return p ? *p : d;
}

// Host: range of Section 4.2's filter threshold (0 = no filter).
inline bool s0_ok(int32_t s0) { return s0 >= 0 && s0 <= 30000; }

__device__ __forceinline__ int seed_key(int a0, int a1, int a2, int a3) {
  // Key = ((c1 * 2 + c2) * 11 + c3) * 20 + c4; -1 when a letter is a stop or
  // the sentinel.
  if ((a0 | a1 | a2 | a3) < 0 || a0 >= NAA || a1 >= NAA || a2 >= NAA || a3 >= NAA) return -1;
  return ((a0 * 2 + c_cls2[a1]) * 11 + c_cls3[a2]) * 20 + a3;
}

}  // namespace plast

// ---------------------------------------------------------------------------
// Library-internal launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
namespace plast {

// prims.cu
void note_launch();  // counts every kernel launch of the library
long long launch_total();
cudaError_t upload_tables_once();
// n_dev (optional, device): the actual element count, at most n; the grids
// are sized for n so the launches need no host copy of the count.
cudaError_t scan_exclusive(const int32_t* in, int64_t* out, int64_t n, int64_t* d_total, void* tmp,
                           size_t tmp_bytes, cudaStream_t st, const int64_t* n_dev = nullptr);
size_t scan_tmp_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                             int bits, void* tmp, size_t tmp_bytes, cudaStream_t st, bool* result_in_alt,
                             const int64_t* n_dev = nullptr);
size_t radix_tmp_bytes(int64_t n);

}  // namespace plast
