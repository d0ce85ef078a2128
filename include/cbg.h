/*
 * cbg.h -- C ABI of a GB300-native (sm_103a) library for the data-parallel hot
 * path of CatBoost training, classic (non-ordered) boosting scheme, as defined in
 * "CatBoost: gradient boosting with categorical features support"
 * (Dorogush, Ershov, Gulin; arXiv 1810.11363).
 *
 * The path: ordered target statistics for categorical features (Section 2,
 * Eq. 1); quantisation of every feature into uint8 bins (Section 5, "Dense
 * numerical features"); per-(leaf, feature, bin) gradient/hessian histograms
 * and L2-regularised split search for oblivious trees (Sections 3 and 5); leaf
 * values, per-row leaf index and the prediction update (Section 3, Section 4
 * "Fast scorer").
 *
 * Conventions shared by every call
 *  - Pointers named as device arrays are CUDA device pointers on the context's
 *    device, owned by the caller; the library never frees them. Pointers named
 *    as host values are plain host memory.
 *  - Every call returns a cbg_status: CBG_OK (0) or a negative error code.
 *    Argument errors are detected on the host before anything is launched and
 *    return CBG_EINVAL. cbg_last_error() gives a message for the last failure.
 *  - Calls are asynchronous on the context's stream (launch order is stream
 *    order); an error raised by a kernel after launch surfaces at the next
 *    cbg_sync() or *_to_host helper. No call synchronises the host except
 *    cbg_sync() and the helpers that say so.
 *  - Layouts: float features and categorical ids are column-major ([F][n]).
 *    Quantised bins use a grouped layout: features are taken 32 at a time and
 *    feature f of row r is the byte at ((f / 32) * n + r) * 32 + f % 32, so one
 *    32-feature group of one row is one 32-byte sector. F_pad (a multiple of 32)
 *    is the padded feature count; bytes of features F..F_pad-1 must be zero. An
 *    optional column-major copy bins_t [F][n] speeds up the per-level leaf update.
 *  - Rows are indexed with int64_t n, 1 <= n <= 2^31 - 1.
 */
#ifndef CBG_H
#define CBG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cbg_status;
#define CBG_OK 0
#define CBG_EINVAL (-1)       /* bad argument, detected on the host          */
#define CBG_ENOMEM (-2)       /* workspace or state buffer too small          */
#define CBG_ECUDA (-3)        /* a CUDA runtime call failed                   */
#define CBG_ETIMEOUT (-4)     /* a bounded device-side wait ran out           */
#define CBG_EUNSUPPORTED (-5) /* valid request this build does not implement  */
#define CBG_EDATA (-6)        /* a device-side data check failed (NaN, range) */

enum { CBG_LABEL_BINARY = 0, CBG_LABEL_REAL = 1 };
enum { CBG_LOSS_RMSE = 0, CBG_LOSS_LOGLOSS = 1 };
enum { CBG_F32 = 0, CBG_BF16 = 1 };

typedef struct cbg_ctx cbg_ctx;

/* One level of an oblivious tree (Section 4 "Fast scorer": one split per
 * level). A row goes to the "1" side iff its bin of `feature` is > `border`.
 * feature = -1 means no candidate existed (every row stays on the "0" side). */
typedef struct cbg_split {
  int32_t feature;
  int32_t border;
  double score;
} cbg_split;

/* Histogram tiling. slab_chunks: 16-feature chunks per work item (2);
 * rows_per_item: rows per CTA of a work unit; threads: threads per histogram
 * CTA (a multiple of 32, <= 512; for the warp-private kernel an upper bound on
 * its warps, each of which holds a private histogram); blocks_per_sm: unused
 * (the grid is sized by the occupancy of clusters); cluster: CTAs per
 * thread-block cluster that share one partial histogram through distributed
 * shared memory (1..16; a smaller power of two is used if that many cannot be
 * co-resident); kernel: 1 = one shared histogram per CTA updated with
 * shared-memory float reductions, 2 = warp-private histograms of 16 features
 * updated without atomics, 3 = one shared histogram per CTA with (G, H)
 * updated by one 64-bit compare-and-swap, 4 = lane-per-feature warp-private
 * histograms with store forwarding (bins must be 16-byte aligned), 5 = the
 * same with G and H in separate warps, 6 = lane-per-feature over the 4-bit
 * packed bins of cbg_pack_bins4 (max_bins <= 16; the level arguments carry
 * bins4), 7 = one shared histogram per CTA of int32 fixed-point cells updated
 * with shared-memory integer reductions (4096 rows per CTA and clusters of 4 by
 * default), 8 = kernel 4 with loader warps: each histogram warp has a partner
 * warp that stages its rows' bin records and (g, h), so that it only updates its
 * histogram (threads counts both; bins 16-byte aligned), 9 = binary features
 * over the 1-bit packed bins of cbg_pack_bits1 (max_bins <= 2; the level
 * arguments carry bits1; 512-thread CTAs whatever threads says). The default (0) is kernel 1, whose shared-memory
 * accumulation is FP32.
 * Kernel 7 is an opt-in form that does not accumulate in FP32: it rounds each (g, h) of a CTA's rows to a
 * multiple of 2^-e, e the largest exponent with 2^e * 1.001 * S < 2^30 for S the
 * sum of |g| (of |h| for H) over those rows, with a dither hashed from the row's
 * position (floor(v 2^e + u), u in [0, 1)): the rounding error of a row is below
 * 2.002 * S * 2^-30 with mean zero (integer values are exact), the sums are exact
 * and do not depend on the order of the updates, and each cluster's cells are
 * rounded once to the FP32 partial. Its error per cell is therefore bounded by the
 * cell's rows times that per-row bound, not by a fraction of the cell's own sum of |g|.
 * cbg_boost_batched batches only kernel 1. Zero fields take library defaults. */
typedef struct cbg_tiles {
  int32_t slab_chunks;
  int32_t rows_per_item;
  int32_t threads;
  int32_t blocks_per_sm;
  int32_t cluster;
  int32_t kernel;
} cbg_tiles;

/* Shape of one boosting problem's tree state. */
typedef struct cbg_tree_shape {
  int64_t n;           /* rows                                   */
  int32_t F;           /* features (floats + one TS column per categorical) */
  int32_t F_pad;       /* padded feature count of bins, multiple of 32, >= F */
  int32_t max_bins;    /* max over features of n_borders + 1, 2..256 (1 allowed: no split) */
  int32_t max_depth;   /* 1..10                                  */
  cbg_tiles tiles;     /* histogram tiling (zero fields = defaults) */
} cbg_tree_shape;

/* ------------------------------------------------------------ context ---- */

/* Create a context on `device` using `cuda_stream` (a cudaStream_t, or NULL for
 * the legacy default stream). `workspace_bytes` preallocates library scratch for
 * the one-off steps (sorts and scans); 0 lets the library grow it on demand
 * (growth is refused with CBG_ENOMEM while the stream is being captured). */
cbg_status cbg_ctx_create(int device, void* cuda_stream, size_t workspace_bytes, cbg_ctx** out);
void cbg_ctx_destroy(cbg_ctx* ctx);
/* Message of the last failure on this context ("" if none). Never NULL. */
const char* cbg_last_error(const cbg_ctx* ctx);
/* Wait for the context's stream; returns CBG_ECUDA / CBG_EDATA / CBG_ETIMEOUT
 * if an asynchronous failure was recorded, else CBG_OK. */
cbg_status cbg_sync(cbg_ctx* ctx);
/* Test hook for the bounded device-side waits (no counterpart in the paper). While
 * enabled (enable != 0), rounds that cbg_boost_batched captures make each wait of its
 * persistent per-level kernel look for a count that can never arrive, and histogram
 * launches of the loader-warp kernel (tiles.kernel 8) have their loaders skip the
 * hand-over of every buffer, so that the compute warps wait for data that never comes.
 * Either kernel gives up after a short limit (about a millisecond per wait) instead of
 * the regular one (about a second): it records a timeout, skips the work behind the
 * wait and ends, and the next cbg_sync returns CBG_ETIMEOUT. The results of such calls
 * are meaningless; the context stays usable. Off by default; not for production use. */
cbg_status cbg_test_force_wait_timeout(cbg_ctx* ctx, int enable);
cbg_status cbg_set_stream(cbg_ctx* ctx, void* cuda_stream);
/* Number of SMs of the context's device (for tiling decisions). */
int cbg_num_sms(const cbg_ctx* ctx);
/* Library version string. */
const char* cbg_version(void);

/* ------------------------------------------------------- preprocessing ---- */

/* The random permutation sigma of Section 2 (before Eq. 1). perm[p] is the row
 * placed at position p: rows sorted by (k_i, i) with k_i the i-th output of a
 * SplitMix64 generator seeded with `seed` (the paper names no generator).
 * perm: device uint32 [n]. */
cbg_status cbg_make_permutation(cbg_ctx* ctx, uint64_t seed, int64_t n, uint32_t* perm);

/* Prior P of Eq. 1 (Section 2): the positive rate for binary labels, the mean
 * label for real labels, computed in FP64 and written to the device double
 * `prior_out`. y: device float [n]; binary labels must be exactly 0 or 1. */
cbg_status cbg_prior(cbg_ctx* ctx, const float* y, int64_t n, int label_kind, double* prior_out);

/* Ordered target statistics, Eq. 1 (Section 2), for C categorical columns:
 * the row at position p of sigma gets (S + a*P) / (N + a), where N and S are the
 * count and label sum of the earlier rows of sigma with the same category.
 * cat: device uint32 [C][n] (any 32-bit ids); y: device float [n]; perm: device
 * uint32 [n] (sigma); prior P and weight a > 0 are host doubles. Outputs in row
 * order: ts device float [C][n] (required); cnt_before device uint32 [C][n] and
 * sum_before [C][n] (uint32 for BINARY labels, double for REAL labels)
 * optional (NULL). N and binary S are exact integers; real S is an FP64
 * segmented prefix sum. (S + a*P)/(N + a) is evaluated in FP64 without
 * fused multiply-add and rounded to float. */
cbg_status cbg_ordered_ts(cbg_ctx* ctx, const uint32_t* cat, const float* y, int64_t n, int32_t C,
                          const uint32_t* perm, double prior, double a, int label_kind, float* ts,
                          uint32_t* cnt_before, void* sum_before);

/* Quantile borders per feature (Section 5: a fixed number of bins per feature,
 * at most 255): v = column f sorted ascending; candidate k = 1..max_borders is
 * v[floor(k*n/(max_borders+1))]; the strictly increasing candidates below max(v)
 * are kept (a -0.0 border is stored as +0.0). x: device float [F][n];
 * borders: device float [F][max_borders] (unused tail set to +inf);
 * n_borders: device int32 [F]. max_borders in 1..254. A NaN or infinity in x
 * makes the next cbg_sync() return CBG_EDATA. */
cbg_status cbg_select_borders(cbg_ctx* ctx, const float* x, int64_t n, int32_t F,
                              int32_t max_borders, float* borders, int32_t* n_borders);

/* Quantisation (Section 5): bin = number of borders strictly below x, written
 * as uint8 to feature f_offset + f of row r of bins (grouped layout, F_pad a
 * multiple of 32) and, if bins_t is not NULL, to bins_t[f_offset + f][r]
 * (column-major, row stride n).
 * x: device float [F][n]; borders / n_borders as from cbg_select_borders.
 * Columns outside [f_offset, f_offset+F) are not touched. */
cbg_status cbg_quantize(cbg_ctx* ctx, const float* x, int64_t n, int32_t F, const float* borders,
                        const int32_t* n_borders, int32_t max_borders, uint8_t* bins, int32_t F_pad,
                        int32_t f_offset, uint8_t* bins_t);

/* ------------------------------------------------------------ boosting ---- */

/* Gradients of the loss at pred (Section 3, Algorithm 1: g = dLoss/da):
 * RMSE g = pred - y, h = 1; Logloss p = 1/(1+exp(-pred)), g = p - y,
 * h = p(1-p). Computed in FP32 and stored as float (CBG_F32) or bfloat16 with
 * round-to-nearest-even (CBG_BF16) into g, h (device [n]). */
cbg_status cbg_gradients(cbg_ctx* ctx, int loss, const float* y, const float* pred, int64_t n,
                         int gh_dtype, void* g, void* h);

/* Bytes of device scratch one tree build needs for `shape` (after tile
 * defaults are applied). */
cbg_status cbg_tree_state_bytes(const cbg_tree_shape* shape, size_t* bytes);

/* Start a tree: every row in leaf 0. state: device scratch of at least
 * cbg_tree_state_bytes(shape) bytes, 256-byte aligned, owned by the caller and
 * reused for every level of the tree; leaf: device uint16 [n], set to 0. */
cbg_status cbg_tree_begin(cbg_ctx* ctx, const cbg_tree_shape* shape, void* state,
                          size_t state_bytes, uint16_t* leaf);

/* Arguments of one level of greedy oblivious-tree growth. */
typedef struct cbg_level_args {
  const cbg_tree_shape* shape; /* host pointer                              */
  void* state;                 /* device scratch from cbg_tree_begin         */
  size_t state_bytes;
  const uint8_t* bins;         /* device, grouped layout (see above)         */
  const uint8_t* bins_t;       /* device [F][n] or NULL                      */
  const int32_t* n_borders;    /* device int32 [F]; candidates k < n_borders[f] */
  const void* g;               /* device [n] gradients (gh_dtype)            */
  const void* h;               /* device [n] hessians (gh_dtype)             */
  int32_t gh_dtype;            /* CBG_F32 or CBG_BF16                        */
  int32_t depth;               /* level d, 0 <= d < max_depth; levels run in order */
  double l2;                   /* L2 regularisation lambda >= 0              */
  int32_t force_feature;       /* >= 0: take this split instead of the best  */
  int32_t force_border;
  uint16_t* leaf;              /* device [n] in/out: leaf += 2^d [bin > k]   */
  cbg_split* splits;           /* device [max_depth]: splits[d] is written   */
  double* child_totals;        /* device [2^(d+1)][2]: (G, H) of every child */
  double* hist_out;            /* optional device [2^d][F][max_bins][2] FP64 */
  int32_t last_level;          /* nonzero: skip re-partitioning the rows     */
  /* Optional challenger: a split on a column outside bins (a feature combination,
   * Section 2). When challenger (device cbg_split) is not NULL and its feature is
   * >= 0, it replaces the best split of bins if its score is strictly higher (or if
   * bins has no candidate). Its feature must be >= F (it names the column, e.g. F + j
   * for the j-th combination of the tree); its border k sends rows with
   * challenger_bins[row] > k to the "1" side (challenger_bins: device uint8 [n], row
   * order), and its FP64 histogram over the 2^d leaves of the level,
   * challenger_hist (device double [2^d][challenger_max_bins][2]), gives the child
   * totals. Ignored when force_feature >= 0. */
  const cbg_split* challenger;
  const uint8_t* challenger_bins;
  const double* challenger_hist;
  int32_t challenger_max_bins;
  /* 4-bit packed bins of the same rows (cbg_pack_bins4), read by the histogram when
   * shape->tiles.kernel is 6; NULL otherwise. */
  const uint8_t* bins4;
  /* 1-bit packed bins of the same rows (cbg_pack_bits1), read by the histogram when
   * shape->tiles.kernel is 9; NULL otherwise. */
  const uint32_t* bits1;
} cbg_level_args;

/* One level d (Sections 3-4): FP64 histograms hist[l][f][b] = sum of (g, h)
 * over rows of leaf l with bin b of feature f, for all 2^d leaves (FP32
 * accumulation in shared memory, FP64 across blocks; one sibling of each pair
 * is obtained by subtracting the other from the parent); the split (f, k)
 * maximising sum_l G_L^2/(H_L+l2) + G_R^2/(H_R+l2) (terms with a zero
 * denominator count as 0; ties to the smallest f, then k); the leaf update
 * leaf += 2^d [bin_f > k]; the child totals; and the row partition used by the
 * next level. */
cbg_status cbg_build_level(cbg_ctx* ctx, const cbg_level_args* args);

/* Leaf values and prediction update (Section 3 leaf values as Newton steps;
 * Section 4 "Fast scorer" leaf index): v_l = -G_l/(H_l + l2) (0 when the
 * denominator is 0) from leaf_totals (device double [2^depth][2]), or taken
 * from leaf_values_in (device double [2^depth]) when leaf_totals is NULL;
 * leaf_r = sum_i 2^i [bins[r][f_i] > k_i] from splits (device [depth]) unless
 * leaf_in (device uint16 [n]) is given; pred_r += float(lr * v_{leaf_r}) (pred
 * device float [n], in/out; lr * v in FP64, the add in FP32). Optional outputs: leaf_out
 * (device uint16 [n]), leaf_values_out (device double [2^depth], v before lr).
 * If y, g and h are not NULL the gradients of `loss` at the updated pred are
 * written to g, h in gh_dtype (fused next-tree gradients). */
typedef struct cbg_apply_args {
  const uint8_t* bins;
  int64_t n;
  int32_t F_pad;
  const cbg_split* splits;
  int32_t depth;
  const double* leaf_totals;
  const double* leaf_values_in;
  double l2;
  double lr;
  const uint16_t* leaf_in;
  uint16_t* leaf_out;
  float* pred;
  double* leaf_values_out;
  const float* y;
  int32_t loss;
  int32_t gh_dtype;
  void* g;
  void* h;
} cbg_apply_args;
cbg_status cbg_apply_tree(cbg_ctx* ctx, const cbg_apply_args* args);

/* Whole boosting run on one problem: T trees of depth D from the current pred
 * (device float [n], in/out). Per tree: gradients (fused into the previous
 * tree's apply), D levels of cbg_build_level, cbg_apply_tree. When use_graph is
 * nonzero one tree is captured as a CUDA graph and replayed. Model outputs:
 * splits device cbg_split [T][D], leaf_values device double [T][2^D] (v before
 * lr). g, h: device scratch [n] of gh_dtype; leaf: device uint16 [n];
 * state: tree-state scratch. */
typedef struct cbg_boost_args {
  const cbg_tree_shape* shape;
  void* state;
  size_t state_bytes;
  const uint8_t* bins;
  const uint8_t* bins_t;
  const int32_t* n_borders;
  const float* y;
  int32_t loss;
  int32_t gh_dtype;
  int32_t depth;
  int32_t trees;
  double lr;
  double l2;
  float* pred;
  void* g;
  void* h;
  uint16_t* leaf;
  cbg_split* splits;
  double* leaf_values;
  double* child_totals;   /* device [2^depth][2] scratch */
  int32_t use_graph;
  const uint8_t* bins4;        /* device 4-bit packed bins or NULL (tiles kernel 6 needs them) */
  const uint32_t* bits1;       /* device 1-bit packed bins or NULL (tiles kernel 9 needs them) */
} cbg_boost_args;
cbg_status cbg_boost(cbg_ctx* ctx, const cbg_boost_args* args);

/* One independent boosting problem of a batched run: its own data, tree state
 * and model outputs (the same arrays as cbg_boost_args). */
typedef struct cbg_problem {
  cbg_tree_shape shape;
  void* state;
  size_t state_bytes;
  const uint8_t* bins;
  const uint8_t* bins_t;
  const int32_t* n_borders;
  const float* y;
  int32_t loss;
  int32_t reserved;
  float* pred;
  void* g;
  void* h;
  uint16_t* leaf;
  cbg_split* splits;       /* device [T][depth] */
  double* leaf_values;     /* device [T][2^depth] */
  double* child_totals;    /* device [2^depth][2] */
} cbg_problem;

/* Batched boosting of many independent problems (each follows cbg_boost, the
 * classic scheme of Sections 3-4); not in the paper. One round -- one tree of every
 * problem -- is captured once as a CUDA graph and replayed `trees` times.
 * When every problem uses the shared-reduction histogram kernel (tiles.kernel 0 or 1)
 * with the same tiling, each step of a round is one launch over all problems: the tree
 * start, then per level one persistent launch whose clusters take histogram work items
 * and FP64 reduction blocks of every problem from one device queue (a reduction block
 * waits, bounded, for its leaf's histogram items: CBG_ETIMEOUT at the next cbg_sync if
 * a wait runs out), then scoring, partition flags and scatter, and the apply and record
 * kernels. Otherwise every problem's tree runs on one of `branches` parallel graph
 * branches (problems round-robin, 0 = min(n_problems, 32)). Every problem uses the same
 * depth, lr, l2 and gradient storage; problem i's result is the same as cbg_boost on it
 * alone (bit for bit where the histogram accumulation order allows; within the tests'
 * tolerances always). problems is a host array. */
cbg_status cbg_boost_batched(cbg_ctx* ctx, const cbg_problem* problems, int32_t n_problems, int32_t gh_dtype,
                             int32_t depth, int32_t trees, double lr, double l2, int32_t branches);

/* ---------------------------------------------------- allocation-free ---- */

/* Histogram of the root leaf (every row) without allocating anything; the paper
 * has no counterpart of this call. It is for callers that cannot allocate device
 * memory: code running inside a host application that owns the whole device
 * memory budget (a framework's caching allocator or a fixed arena) and plugin
 * code that may not call cudaMalloc. cbg_build_level needs a caller-allocated
 * tree state; this call needs only its inputs and its output and makes no
 * cudaMalloc, cudaFree or other allocating call.
 *
 * Result: hist_out (device double [F][max_bins][2]) holds, for every feature f
 * and bin b, the FP64 sums of g and h over all rows whose bin of f is b, the
 * same values cbg_build_level writes to hist_out at depth 0. bins, g, h are as
 * for cbg_build_level (grouped bins layout; g, h of gh_dtype).
 *
 * Scratch: a file-scope device array of 16 MiB (the work plan and the FP32
 * partial histograms), held by every GPU that loads the library until the
 * process exits. One work unit needs F_pad/32 * max_bins * 256 bytes, so
 * F_pad * max_bins beyond about 2 million is rejected with CBG_EINVAL. Rows are
 * split over as many units as the array holds; a CTA of a unit then sums up to
 * 16384 rows into its FP32 histogram (the accuracy of the other paths: within
 * 1e-5 of each bin's sum of |g|), and an n that would need more rows per CTA
 * is rejected with CBG_EINVAL (for example F_pad 2048 at 128 bins holds about
 * 9e5 rows, F_pad 96 at 255 bins about 1.1e7). n must be at most 2^31 - 2^20.
 * The first call through a context looks up the array's device address (once
 * per device and context, with that device current): make that first call
 * before any stream capture. Every call shares the array and overwrites
 * what the previous call left there, so calls that can overlap on the GPU (on
 * different streams, or from different contexts on the same device) race: order
 * them on one stream or serialise them. */
cbg_status cbg_histogram_noalloc(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F, int32_t F_pad,
                                 int32_t max_bins, const void* g, const void* h, int32_t gh_dtype,
                                 double* hist_out);

/* ------------------------------------------------------------ profiling ---- */

/* Device-time accounting of the histogram kernel: while enabled, a pair of CUDA
 * events is recorded on the context stream around every histogram launch.
 * cbg_profile_read synchronises the stream and returns the summed device time
 * (milliseconds) and the number of launches since the last reset (reset != 0
 * clears both afterwards). Not available while the stream is being captured. */
cbg_status cbg_profile_enable(cbg_ctx* ctx, int enable);
cbg_status cbg_profile_read(cbg_ctx* ctx, int reset, double* hist_ms, int64_t* hist_launches);

/* Rows read by histogram launches (rows of the leaves histogrammed directly,
 * summed over levels) since the tree state was last reset through this call
 * (reset != 0); synchronises the stream. The state must have been initialised
 * by cbg_tree_begin. */
cbg_status cbg_tree_rows_histogrammed(cbg_ctx* ctx, const cbg_tree_shape* shape, void* state, int reset,
                                      int64_t* rows);

/* ------------------------------------------------------------ inference -- */

/* Full-data target-statistic table of one categorical column, for rows that are
 * not in the training permutation (Section 2, Eq. 1 with every training row
 * counted as seen before the new row). The table lists the distinct category
 * ids ascending, each with the label sum S and the count N over all n training
 * rows.
 * cat: device uint32 [n]; y: device float [n].
 * ids, cnts: device uint32 [n]; sums: device double [n]. The first *n_unique
 * entries are written.
 * n_unique: device int32 [1].
 * Binary-label sums are exact integers; real-label sums are FP64 segmented sums
 * (another order than the row order). Uses the context workspace. */
cbg_status cbg_ts_table(cbg_ctx* ctx, const uint32_t* cat, const float* y, int64_t n, int label_kind,
                        uint32_t* ids, double* sums, uint32_t* cnts, int32_t* n_unique);

/* Target statistic of m new rows from a cbg_ts_table table: a row with
 * category c gets (S_c + a*P) / (N_c + a), evaluated in FP64 without fused
 * multiply-add and rounded to float; a category absent from the table gets
 * (0 + a*P)/(0 + a).
 * ids/sums/cnts/n_unique: device, as written by cbg_ts_table.
 * cat_new: device uint32 [m]; ts: device float [m].
 * prior P and a > 0: host doubles. */
cbg_status cbg_ts_apply(cbg_ctx* ctx, const uint32_t* ids, const double* sums, const uint32_t* cnts,
                        const int32_t* n_unique, const uint32_t* cat_new, int64_t m, double prior, double a,
                        float* ts);

/* Model prediction (Section 4 "Fast scorer"). For every row r, trees t = 0..T-1 in
 * order:
 *   leaf = sum_d 2^d [bin(r, f_td) > k_td]
 *   pred[r] += float(lr * leaf_values[t][leaf])
 * The sum is in FP32 in tree order, the same arithmetic as cbg_apply_tree, so
 * the training rows get back their training predictions bit for bit. A level
 * with feature -1 sends every row to its 0 side.
 * bins_t: device uint8 [F][n] (column-major, as cbg_quantize writes it);
 * splits: device cbg_split [T][depth]; leaf_values: device double [T][2^depth]
 * (before the learning rate); pred: device float [n], in/out (zero it for a
 * fresh prediction). depth 1..10. Uses the context workspace for the per-tree
 * increments float(lr * v). */
typedef struct cbg_predict_args {
  const uint8_t* bins_t;
  int64_t n;
  int32_t F;
  const cbg_split* splits;
  const double* leaf_values;
  int32_t trees;
  int32_t depth;
  double lr;
  float* pred;
} cbg_predict_args;
cbg_status cbg_predict(cbg_ctx* ctx, const cbg_predict_args* args);

/* ------------------------------------------------------------ autotuner -- */

/* Histogram-tile autotuner. The paper has no counterpart: it picks the tiling
 * that the batched form (and any caller) uses for a problem shape.
 * It times a fixed list of candidate tilings on the caller's own data, building
 * `depth` levels of one tree per timing (cbg_tree_begin + cbg_build_level on the
 * ctx stream, CUDA events), and writes the fastest to *best and its mean device
 * time per tree (ms) to *best_ms. The candidates vary:
 *  - the histogram kernel: shared-memory reductions (1), lane-per-feature warp
 *    histograms (4), their loader-warp form (8) and their one-statistic-per-warp
 *    form (5), 16-feature
 *    warp-private histograms (2), with bins4 and max_bins <= 16 the packed
 *    lane-per-feature kernel (6), with bits1 and max_bins <= 2 the 1-bit kernel
 *    (9), and with fixed_point != 0 the fixed-point shared-reduction kernel (7);
 *  - CTAs per cluster;
 *  - rows per CTA of a work unit.
 * Ownership and layout follow cbg_build_level. args->shape->tiles is ignored.
 * state must hold cbg_autotune_state_bytes(shape) bytes; a candidate whose state
 * does not fit, or that the device cannot launch, is skipped. leaf, splits and
 * child_totals are overwritten. reps >= 1 timed trees per candidate, after one
 * untimed. Synchronises the stream. CBG_EINVAL while the stream is being
 * captured or if no candidate ran. */
typedef struct cbg_autotune_args {
  const cbg_tree_shape* shape; /* host pointer; tiles ignored                 */
  void* state;                 /* device scratch, see cbg_autotune_state_bytes */
  size_t state_bytes;
  const uint8_t* bins;         /* device, grouped layout, 16-byte aligned     */
  const uint8_t* bins_t;       /* device [F][n] or NULL                       */
  const int32_t* n_borders;    /* device int32 [F]                            */
  const void* g;               /* device [n] (gh_dtype)                       */
  const void* h;
  int32_t gh_dtype;
  int32_t depth;               /* levels per timed tree, 1..max_depth          */
  double l2;
  uint16_t* leaf;              /* device [n] scratch                          */
  cbg_split* splits;           /* device [max_depth] scratch                  */
  double* child_totals;        /* device [2^depth][2] scratch                 */
  int32_t reps;
  const uint8_t* bins4;        /* device 4-bit packed bins (cbg_pack_bins4) or NULL; with
                                  max_bins <= 16 the packed kernel is a candidate too */
  int32_t fixed_point;         /* nonzero: the fixed-point kernel (7) is a candidate too */
  const uint32_t* bits1;       /* device 1-bit packed bins (cbg_pack_bits1) or NULL; with
                                  max_bins <= 2 the 1-bit kernel (9) is a candidate too */
} cbg_autotune_args;

/* 4-bit packed bins (Section 5 "Dense numerical features": features with at most
 * 15 borders take 4 bits): bins4[q][r][i] holds feature 64q + i of row r in its
 * low nibble and feature 64q + 32 + i in its high nibble (device uint8
 * [ceil(F_pad/64)][n][32], caller-owned, 16-byte aligned like bins). Every bin
 * of bins must be below 16; a larger one makes the next cbg_sync() return
 * CBG_EDATA. The packed records are half the bytes of the grouped layout; the
 * histogram kernel 6 (tiles.kernel) reads them. */
cbg_status cbg_pack_bins4(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F_pad, uint8_t* bins4);

/* 1-bit packed bins (Section 5 "Dense numerical features": binary features take 1
 * bit, 32 features to a 32-bit integer): bit i of bits1[q][r] is 1 when feature
 * 32q + i of row r has bin 1 (device uint32 [F_pad/32][n], caller-owned, 16-byte
 * aligned like bins). Every bin of bins must be 0 or 1; a larger one makes the
 * next cbg_sync() return CBG_EDATA. A row's 32 features take 4 bytes instead of
 * 32; the histogram kernel 9 (tiles.kernel) reads them. */
cbg_status cbg_pack_bits1(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F_pad, uint32_t* bits1);

/* Tree-state bytes large enough for every autotuner candidate of `shape`. */
cbg_status cbg_autotune_state_bytes(const cbg_tree_shape* shape, size_t* bytes);
cbg_status cbg_autotune_tiles(cbg_ctx* ctx, const cbg_autotune_args* args, cbg_tiles* best, double* best_ms);

/* ------------------------------------------------- ordered boosting ---- */
/* Ordered boosting (Section 3 "Fighting Gradient Bias", Algorithm 1, with the
 * log-scale supporting models M'_i and tree structures shared by all models).
 *
 * There are s permutations sigma_q (position -> row). Each has its own bins: the
 * float columns are shared and the categorical columns hold the ordered TS
 * computed along sigma_q, quantised with one set of borders. Every permutation's
 * data is kept in its own position order (cbg_permute_rows).
 *
 * Supporting values of one permutation: cbg_ordered_sup_len(n) floats, the
 * 2^(I+1) + n used ones (I = floor(log2(n-1)), I = 0 for n = 1) rounded up to a
 * multiple of 64; sup is [s][cbg_ordered_sup_len(n)]. Model M'_i,
 * i = 0..I, is trained on positions p < 2^i and holds positions
 * j < min(2^(i+1), n), position j at element 2^(i+1) + j (the last model at
 * 2^(I+1) + j); elements 0 and 1 are unused. A fresh run starts from zeros. */
cbg_status cbg_ordered_sup_len(int64_t n, int64_t* len);

/* Bytes of the device work buffer cbg_boost_ordered needs (leaf indices of every
 * permutation and FP64 leaf totals). */
cbg_status cbg_ordered_work_bytes(int64_t n, int32_t s, int32_t depth, size_t* bytes);

/* Rows into the position order of perm (device uint32 [n], position -> row):
 * bins_pos[g][k][.] = bins[g][perm[k]][.] in the grouped layout (F_pad a
 * multiple of 32, both 16-byte aligned), bins_t_pos[f][k] = bins_t[f][perm[k]]
 * ([F][n]), y_pos[k] = y[perm[k]]. Each input may be NULL to skip it; outputs
 * are device buffers of the same sizes, owned by the caller. */
cbg_status cbg_permute_rows(cbg_ctx* ctx, const uint32_t* perm, int64_t n, int32_t F, int32_t F_pad,
                            const uint8_t* bins, const uint8_t* bins_t, const float* y, uint8_t* bins_pos,
                            uint8_t* bins_t_pos, float* y_pos);

/* Arguments of cbg_boost_ordered. All pointers are device memory except shape. */
typedef struct cbg_ordered_args {
  const cbg_tree_shape* shape; /* n, F, F_pad, max_bins, max_depth, tiles      */
  void* state;                 /* tree-state scratch (cbg_tree_state_bytes)    */
  size_t state_bytes;
  int32_t s;                   /* permutations, >= 1                           */
  const uint8_t* bins_pos;     /* [s][F_pad/32][n][32]: permutation q's bins in its position order */
  const uint8_t* bins_t_pos;   /* [s][F][n] the same, per feature, or NULL     */
  const float* y_pos;          /* [s][n] labels in each position order         */
  const uint8_t* bins;         /* grouped, row order: the final model's bins (permutation 0's) */
  const uint8_t* bins_t;       /* [F][n] row order, or NULL                    */
  const int32_t* n_borders;    /* [F]                                          */
  const float* y;              /* [n] row order                                */
  int32_t loss;                /* CBG_LOSS_RMSE or CBG_LOSS_LOGLOSS            */
  int32_t gh_dtype;            /* storage of the ordered gradients             */
  int32_t depth;
  int32_t trees;
  int32_t first_tree;          /* tree t of the call takes permutation (first_tree + t) mod s */
  double lr;
  double l2;
  float* pred;                 /* [n] row order, in/out: the final model       */
  float* sup;                  /* [s][cbg_ordered_sup_len(n)] in/out           */
  void* g;                     /* [n] scratch of gh_dtype                      */
  void* h;
  uint16_t* leaf;              /* [n] scratch                                  */
  cbg_split* splits;           /* [trees][depth] out                           */
  double* leaf_values;         /* [trees][2^depth] out, v before lr            */
  double* child_totals;        /* [2^depth][2] scratch                         */
  void* work;                  /* cbg_ordered_work_bytes(n, s, depth) bytes    */
  size_t work_bytes;
  int32_t use_graph;           /* nonzero: after the first tree, replay one captured tree per permutation */
} cbg_ordered_args;

/* `trees` iterations of ordered boosting. Tree t (permutation r = (first_tree +
 * t) mod s):
 *  1. ordered gradients: position k >= 1 of sigma_r at M'_{r,floor(log2 k)}(x_k),
 *     position 0 at the start value 0 (stored in gh_dtype, position order);
 *  2. the structure: cbg_build_level for every level on permutation r's bins;
 *  3. the final model (the second phase, done the classic way): leaf indices on
 *     `bins`, FP64 totals of the plain gradients at pred, v = -G/(H+l2),
 *     pred += float(lr v);
 *  4. every supporting model of every permutation: leaf indices on its
 *     permutation's bins, FP64 totals of the gradients at its own values over its
 *     training positions, v = -G/(H+l2) (0 when H+l2 = 0), and float(lr v) added
 *     at every position it holds.
 * Gradients are computed in FP32. */
cbg_status cbg_boost_ordered(cbg_ctx* ctx, const cbg_ordered_args* args);

/* ---------------------------------------------- feature combinations ---- */
/* Greedy categorical feature combinations (Section 2 "Feature combinations";
 * Section 5 "Categorical features").
 *
 * An item is a categorical column or a split already taken in the tree; a
 * combination is a set of items. kind 0: categorical column a (its ids, b = 0);
 * kind 1: the two-valued column [bin of feature a > b]. Items are kept sorted by
 * (kind, a, b). A combination's value in a row is the SplitMix64 chain
 * h <- splitmix64(seed = h, index = v) over its items in that order from h = 0
 * (v = the id, or the bit), folded to 32 bits as h ^ (h >> 32); it is converted
 * to a number by Eq. 1 along perm (prior and a as for single columns) and
 * quantised with max_borders borders chosen on that column (the border rule of
 * cbg_select_borders). */
typedef struct cbg_combo_item {
  int32_t kind;   /* 0 categorical column, 1 split; -1 marks an unused slot */
  int32_t a;
  int32_t b;
} cbg_combo_item;

/* Values of one combination for n rows (device uint32 ids [n]): items (host,
 * n_items of them, 1..16, sorted by (kind, a, b) without repeats) over cat
 * (device uint32 [C][n], kind 0) and bins_t (device uint8 [F][n], kind 1). The
 * same chain as the training path, for applying a combination split to new rows
 * (with cbg_ts_table / cbg_ts_apply / cbg_quantize). Synchronises the stream. */
cbg_status cbg_combo_ids(cbg_ctx* ctx, const cbg_combo_item* items, int32_t n_items, const uint32_t* cat, int32_t C,
                         const uint8_t* bins_t, int32_t F, int64_t n, uint32_t* ids);

/* Bytes of the device work buffer of cbg_boost_combos. */
cbg_status cbg_combo_work_bytes(int64_t n, int32_t C, int32_t depth, int32_t max_borders, int32_t max_complexity,
                                size_t* bytes);

/* Arguments of cbg_boost_combos. Device memory unless marked host. */
typedef struct cbg_combo_args {
  const cbg_tree_shape* shape; /* host; shape->F = F_float + C             */
  void* state;                 /* tree-state scratch (cbg_tree_state_bytes) */
  size_t state_bytes;
  const uint8_t* bins;         /* grouped: F_float floats, then one TS column per categorical */
  const uint8_t* bins_t;       /* [F][n], required (splits joined as items)   */
  const int32_t* n_borders;    /* [F]                                         */
  const uint32_t* cat;         /* [C][n] raw category ids                     */
  int32_t C;
  int32_t F_float;
  const uint32_t* perm;        /* [n] sigma, position -> row (Eq. 1)          */
  const float* y;              /* [n]                                         */
  int32_t label_kind;          /* CBG_LABEL_BINARY or CBG_LABEL_REAL          */
  int32_t max_borders;         /* borders of a combination's column, 1..254   */
  double prior;
  double a;                    /* prior weight of Eq. 1                       */
  int32_t max_complexity;      /* items per combination, 1..16 (1: none)      */
  int32_t loss;
  int32_t gh_dtype;
  int32_t depth;
  int32_t trees;
  int32_t reserved;
  double lr;
  double l2;
  float* pred;                 /* [n] in/out                                  */
  void* g;                     /* [n] scratch of gh_dtype                     */
  void* h;
  uint16_t* leaf;              /* [n] scratch                                 */
  cbg_split* splits;           /* [trees][depth] out; a combination is F + j  */
  double* leaf_values;         /* [trees][2^depth] out                        */
  double* child_totals;        /* [2^depth][2] scratch                        */
  void* work;                  /* cbg_combo_work_bytes(...) bytes             */
  size_t work_bytes;
  cbg_combo_item* combo_items; /* host [trees][depth][max_complexity] out: the combination of a
                                  combination split, kind -1 elsewhere */
  int32_t* combo_nb;           /* host [trees][depth] out: its border count   */
  float* combo_borders;        /* host [trees][depth][max_borders] out: its borders */
} cbg_combo_args;

/* Classic boosting (as cbg_boost) with greedy feature combinations. The first
 * level of a tree takes no combination. At level d >= 1 the candidates are
 * every item set present in the tree -- {c} for a split on categorical c's TS
 * column, {(f, k)} for a split on float feature f, the combination itself for a
 * combination split -- joined with every categorical column it lacks, up to
 * max_complexity items, without repeats, in lexicographic order of their sorted
 * items. Every candidate's best border is scored on the current leaves like an
 * ordinary feature (Section 3 score); the best (ties to the first candidate,
 * then the smallest border) replaces the best ordinary split only with a
 * strictly higher score. Synchronises the host once per level. */
cbg_status cbg_boost_combos(cbg_ctx* ctx, const cbg_combo_args* args);

#ifdef __cplusplus
}
#endif

#endif /* CBG_H */
