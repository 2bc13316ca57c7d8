// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msm.h"

namespace msm {

constexpr int kMaxWords = 4;    // ell <= 256
constexpr int kMaxBlocks = 32;  // k <= 32 (block sets fit a uint32 mask)
constexpr int kMaxDim = 4096;

// Bit layout of the k blocks of a string of ell symbols of sw bits (sw = 1:
// the sign bits of Eq. 3; sw = 2 or 4: E2LSH symbols), Sec. 2.2: blocks of
// approximately equal length, aligned to symbols.  Passed to kernels by value.
struct BlockLayout {
  int ell, k, W;  // ell: bits (symbols * sw)
  int sw;         // bits per symbol
  int lo[kMaxBlocks];
  int width[kMaxBlocks];
  uint64_t mask[kMaxBlocks][kMaxWords];
};

BlockLayout make_layout(int ell_sym, int k, int sw = 1);

// One grouping (replicate q, kept block set K) of the multiple sorting
// method; the grouping key of a string is its K blocks.
struct MaskDesc {
  uint64_t keep[kMaxWords];  // bits of the kept blocks
  uint32_t K;                // kept blocks as a bit set
  int kept_bits;             // number of kept bits
  int maxK;                  // highest kept block index
  int ngap;                  // blocks below maxK that are not kept
  uint8_t gap[kMaxBlocks];   // those blocks: a pair is reported under K only
                             // if it differs in every one of them
  // Grouping key = (K-block part << sub_width) | value of the first gap
  // block.  Strings equal on that block can never be reported under K, so
  // runs of equal full keys inside a group need no inspection.
  int sub_lo, sub_width;     // first gap block (width 0: no sub-key)
  int hashed;                // K-block part is a mix, not the exact blocks
};

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define MSM_CUDA(call)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::msm::cuda_fail(e_, #call); \
  } while (0)
#define MSM_LAUNCH(what)                                  \
  do {                                                    \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) return ::msm::cuda_fail(e_, what); \
    ::msm::count_launch();                                \
  } while (0)

int num_sms();

// Kernel launch accounting: a process-wide launch counter, and (when a call
// asked for statistics) CUDA events around every launch, summed per class.
enum KernelClass {
  KC_PROJECT = 0, KC_HIST = 1, KC_SCATTER = 2, KC_SCAN = 3,
  KC_BOUNDS = 4, KC_CHECK = 5, KC_RECHECK = 6, KC_OTHER = 7
};
void count_launch();
void kt_begin(int kc, cudaStream_t s);
void kt_end(cudaStream_t s);
struct KernelTimes;
struct KtScope {  // installs a per-call timer for this thread
  explicit KtScope(bool on);
  ~KtScope();
  void collect(float* ms, int64_t* launches);
  KernelTimes* t;
};

// ------------------------------------------------------------ scratch
// Buffers of a reusable execution plan, in the order they were requested.
struct ScratchLog {
  void* ptr[128];
  size_t bytes[128];
  int count = 0;
  int next = 0;   // replay position
};

// Device memory for one call: every buffer comes from the caller's
// allocator (or cudaMallocAsync) and is released, stream-ordered, when the
// Scratch goes out of scope, except buffers handed over with release().
// Plan modes (a ScratchLog): recording allocates and logs every buffer and
// frees nothing (the plan owns them); replaying hands the logged buffers out
// again in the same order, so a captured CUDA graph sees exactly the
// buffers of the recorded run.  Both modes mark the call as sync-free:
// checks that would read a device word back are deferred to the plan.
class Scratch {
 public:
  Scratch(const msm_allocator* a, cudaStream_t s) : a_(a), s_(s) {}
  Scratch(const msm_allocator* a, cudaStream_t s, ScratchLog* log, bool replay)
      : a_(a), s_(s), log_(log), replay_(replay) {}
  ~Scratch();
  void* get(size_t bytes);          // NULL on failure (error message set)
  void put(void* p);                // free now (stream-ordered)
  void release(void* p);            // hand ownership to the caller
  cudaStream_t stream() const { return s_; }
  const msm_allocator* allocator() const { return a_; }
  bool sync_free() const { return log_ != nullptr; }
  bool replaying() const { return replay_; }
 private:
  const msm_allocator* a_;
  cudaStream_t s_;
  void* live_[64];
  int nlive_ = 0;
  ScratchLog* log_ = nullptr;
  bool replay_ = false;
};

void* raw_alloc(const msm_allocator* a, size_t bytes, cudaStream_t s);
void raw_free(const msm_allocator* a, void* p, cudaStream_t s);

// ------------------------------------------------------ kernel launchers
// rng.cu
int launch_gaussian(uint64_t seed, int64_t count, float* out, cudaStream_t s);
// E2LSH bucket offsets in [0, 1) (Philox4x64-10, key {seed, 2}).
int launch_e2lsh_offsets(uint64_t seed, int64_t count, float* out, cudaStream_t s);
// m uniform random pairs i != j of n points (Philox4x64-10, key {seed, 1}).
int launch_random_pairs(uint64_t seed, int64_t m, int64_t n, uint64_t* out, cudaStream_t s);

// project.cu
// Row norms in double (sequential fma of squares, then sqrt) plus a flag
// word: bit 0 = some row has norm 0, bit 1 = some value is not finite.
int launch_row_norms(const void* X, int dtype, int64_t n, int dim,
                     double* nrm64, float* nrm32, unsigned* flags,
                     cudaStream_t s);
int launch_col_norms(const float* R, int Q, int dim, int ell, float* rn,
                     cudaStream_t s);
// E2LSH symbols: low sw bits of floor(r^T x / width + u), strings
// [Q][n][ceil(ell sw / 64)]; rnorm: column norms of R, xnorm: row norms.
int launch_project_e2lsh(const void* X, int dtype, int64_t n, int dim, const float* R,
                         const float* rnorm, const float* xnorm, const float* u, int Q,
                         int ell, int sw, float width, uint64_t* strings,
                         unsigned long long* recompute, cudaStream_t s);
int launch_project(const void* X, int dtype, int64_t n, int dim,
                   const float* R, const float* rnorm, const float* xnorm,
                   int Q, int ell, uint64_t* strings,
                   unsigned long long* recompute, cudaStream_t s);

// project_tc.cu: the same projection on tcgen05 tensor cores (X and R split
// into bf16 high and low parts, three MMAs; bf16 X needs two), TMA-fed,
// sign/pack in the TMEM epilogue; undecided bits are queued and settled by
// a fix-up kernel.
bool tc_project_supported(int dtype, int dim, uintptr_t xaddr);
// Poll limit of the projection's bounded waits (0: the default); returns
// the previous limit.
int set_wait_polls(uint32_t polls);
uint32_t wait_polls();

// mlp_tc.cu: the learned projection's feature map on tcgen05 (both layers
// fused per 128 rows); ws: mlp_tc_scratch_bytes.  Synchronises (reads the
// status of its bounded waits).
bool mlp_tc_supported(int dtype, int dim, int hidden, int dim_out, uintptr_t xaddr);
size_t mlp_tc_scratch_bytes(int64_t n, int dim, int dtype);
int launch_mlp_tc(const void* X, int dtype, int64_t n, int dim, const void* W1,
                  const float* b1, const void* W2, const float* b2, int hidden, int dim_out,
                  float* Y, void* ws, cudaStream_t s);
size_t tc_project_scratch_bytes(int64_t n, int dim, int Q, int ell, int dtype);
// *fell_back = true when the queue overflowed (the caller must then run the
// SIMT projection, which overwrites every string).  fell_back == NULL: no
// host round trip; an overflow is reported in *status bit 1 instead.
int launch_project_tc(const void* X, int dtype, int64_t n, int dim,
                      const float* R, const float* xnorm, int Q, int ell,
                      uint64_t* strings, unsigned long long* recompute,
                      void* ws, unsigned* status, bool* fell_back,
                      cudaStream_t s);

// Point sets of a batched call: set s holds the points [off[s], off[s+1])
// of the pool, and a group (run of equal grouping keys) never spans two
// sets.  A single pool is one set with all pointers NULL.
struct SetTable {
  int S = 1;                            // sets
  const int64_t* off = nullptr;         // device [S+1]
  const int* tile_set = nullptr;        // device [T]: set of each radix tile
  const int* set_tile0 = nullptr;       // device [S+1]: first radix tile of each set
  const uint32_t* start_bits = nullptr; // device bitmap over points: bit p set
                                        // iff some set other than the first
                                        // starts at point p
  int T = 0;                            // radix tiles per grouping segment
};
// Items per radix tile of the grouping sort (tiles never straddle sets).
int group_tile_items();

// group.cu: grouping of every (mask, string) of a batch of masks.
struct GroupBatch {
  const uint64_t* strings;  // the replicate's pool [n][W]
  int64_t n;
  int W;
  const MaskDesc* masks;    // device [S]
  int S;                    // masks in this batch
  int group_bits;           // key width (8..32)
  int passes;               // ceil(group_bits / 8)
  const BlockLayout* layout;  // device copy
  SetTable sets;            // point sets (one set: defaults)
};
size_t group_scratch_bytes(int64_t n, int S, int nsets = 1);
// Sorts (key, index) of all S*n items by key within each mask segment;
// on return keys/vals hold the sorted order (pointers into `ws`).
int run_grouping(const GroupBatch& b, void* ws, uint32_t** keys_out,
                 uint32_t** vals_out, cudaStream_t s);
// Generic exclusive scans (device-wide), returning the total in *total_dev.
size_t scan_scratch_bytes(int64_t len);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t len,
                       void* ws, uint32_t* total_dev, cudaStream_t s);
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, int64_t len,
                       void* ws, uint64_t* total_dev, cudaStream_t s);
// Same, with the length read on the device (min(len_max, *len_dev)).
int exclusive_scan_u64_devlen(const uint64_t* in, uint64_t* out,
                              int64_t len_max, const uint32_t* len_dev,
                              void* ws, uint64_t* total_dev, cudaStream_t s);
// Radix sort of one segment of 64-bit keys with 32-bit payloads (used for
// the canonical order of the output).
size_t sort64_scratch_bytes(int64_t m);
int sort_pairs64(uint64_t* keys, uint32_t* vals, int64_t m, int key_bits,
                 void* ws, cudaStream_t s);

// pairs.cu: group boundaries and the in-group pair check.
// Dense tiles of the pair-list check.  A tile whose passing pairs are many
// is stored as one record instead of one candidate per pair, so that the
// recheck reads the tile's rows once (recheck_tiles in recheck.cu).  Record
// at word offset o of pool: [o] = number of entries | (rows are the columns)
// << 31; [o + 1, o + 33) the row points; [o + 33, o + 65) the column points;
// then the entries (row << 5 | column), two 16-bit entries per word.  offs[r]
// is record r's offset, or kNoRecord when the pool was full (its pairs went to
// the candidate list instead).  ctr: [0] records reserved, [1] pool words
// reserved, [2] pairs stored in records.
constexpr uint32_t kNoRecord = 0xFFFFFFFFu;
constexpr int kRecHeader = 65;
struct TileRecs {
  uint32_t* pool = nullptr;  // NULL: no records, every candidate goes to E
  uint64_t pool_cap = 0;     // words
  uint32_t* offs = nullptr;
  uint32_t cap = 0;          // records
  unsigned long long* ctr = nullptr;
  uint32_t min_pairs = 64;   // a tile with fewer passing pairs appends them to E
};

struct PairBatch {
  const uint32_t* keys;      // sorted keys [S*n]
  const uint32_t* vals;      // point index of each sorted item [S*n]
  const uint64_t* strings;   // all pools [Q][n][W]
  int64_t n;
  int W;
  int S;
  int q;                     // replicate of this batch
  int d;
  int group_bits;            // grouping-key width (keys are exact when the
                             // kept bits fit)
  const MaskDesc* masks;     // device [S]
  const BlockLayout* layout; // device copy
  const uint32_t* fields;    // optional field layout [Q][n][FP] (or NULL)
  int FP;                    // stored words per string (even)
  int FU;                    // words holding fields, ceil(k / 2)
  const uint32_t* start_bits = nullptr;  // set starts (SetTable::start_bits)
  // Fused recheck (count-only output): when X is set, every pair that passes
  // the tests is rechecked against eps at once and counted; nothing is
  // appended to the candidate list.
  const void* X = nullptr;
  int dtype = 0, dim = 0, metric = 0;
  float eps = 0.f;
  const float* nrm = nullptr;            // float row norms (cosine)
  unsigned long long* kept = nullptr;    // [0] pairs within eps,
                                         // [1] double-precision decisions
  unsigned long long* set_kept = nullptr;  // per-set pairs within eps (or NULL)
  const int64_t* set_off = nullptr;      // device [nsets + 1]
  int nsets = 1;
  int sw = 1;                            // bits per symbol (1: sign bits)
  unsigned long long* evaluated = nullptr;  // pairs that took the per-pair
                                           // tests after the prefilter
  TileRecs recs;                         // dense-tile records (pair-list eps graph)
  // launch tuning of the pair check (0 = defaults)
  int ctas_per_sm = 0;
  int min_blocks = 0;                    // fused variant: 2, 4 or 5
};
size_t pairs_scratch_bytes(int64_t items);
// Field layout: every block in its own 16-bit field, FP (even) words per
// string; field_words returns 0 when a block exceeds 15 bits or k > 16.
int field_words(int ell_sym, int k, int sw = 1);
int launch_fields(const uint64_t* strings, int64_t count, int ell_sym, int k, int sw,
                  uint32_t* fields, cudaStream_t s);
// Finds the groups of >= 2 equal keys; returns on the device the number
// of work items and adds sum C(size,2) to *checks_dev.
int find_groups(const PairBatch& b, void* ws, unsigned long long* checks_dev,
                cudaStream_t s);
// Checks every pair of every group and appends the pairs reported under
// this (replicate, mask) to cand (capacity cap) at *count_dev.
int check_groups(const PairBatch& b, void* ws, uint64_t* cand, int64_t cap,
                 unsigned long long* count_dev, cudaStream_t s);

// Per-set pair counts of a finished pair list (counts: device [S], added to).
int launch_set_counts(const uint64_t* pairs, int64_t m, const int64_t* off, int S,
                      unsigned long long* counts, cudaStream_t s);

// mlp.cu: learned projection network
int mlp_forward(const void* X, int dtype, int64_t n, int dim, const void* W1,
                const float* b1, const void* W2, const float* b2, int hidden,
                int dim_out, float* Y, float* Hbuf, float* Abuf, int64_t chunk,
                const uint32_t* rowmap, cudaStream_t s);
int mlp_grad(const void* X, int dtype, int64_t n, int dim, const void* W1,
             const float* b1, const void* W2, const float* b2, int hidden, int dim_out,
             const uint32_t* pi, const uint32_t* pj, const uint8_t* label, int64_t B,
             float m_pos, float m_neg, float* grads, float* loss_dev, void* ws,
             cudaStream_t s);
int mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count,
             int step, float lr, float beta1, float beta2, float eps, void* w1h, void* w2h,
             int hidden, int dim, int dim_out, cudaStream_t s);

// recheck.cu.  bad_dev (optional): set nonzero when some candidate is not a
// pair i < j < n (such candidates are skipped without reading X).
int launch_recheck(const void* X, int dtype, int64_t n, int dim, int metric,
                   float eps, const float* nrm32, const uint64_t* cand,
                   const unsigned long long* m_dev, int64_t m_max,
                   uint64_t* pairs_out, float* dist_out,
                   unsigned long long* count_dev,
                   unsigned long long* recompute_dev, unsigned* bad_dev,
                   cudaStream_t s);
// The recheck of the dense-tile records 0 .. nrec - 1 (offsets in recs.offs),
// appending kept pairs and distances after those already in the output.
int launch_recheck_tiles(const void* X, int dtype, int64_t n, int dim, int metric, float eps,
                         const float* nrm32, const TileRecs& recs, uint32_t nrec,
                         uint64_t* pairs_out, float* dist_out, unsigned long long* count_dev,
                         unsigned long long* recompute_dev, cudaStream_t s);
// Whether rows of this shape can be staged whole by recheck_tiles.
bool tile_recheck_supported(const void* X, int dtype, int dim);
int launch_eps_count(const void* X, int dtype, int64_t n, int dim, int metric,
                     float eps, const float* nrm32,
                     unsigned long long* count_dev, cudaStream_t s);

}  // namespace msm
