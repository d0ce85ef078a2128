// CPU oracle for the CatBoost training hot path (arXiv 1810.11363).
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded
// restatement of what the method computes, in FP64 unless a step fixes the
// storage precision. It exists so that tests, the smoke check and the CPU
// baseline of the benchmark can compare the CUDA library against something
// obviously correct. Nothing in the product path may link, load or call it, and
// it shares no code with the CUDA sources.
//
// Built with -ffp-contract=off so that no multiply-add is fused: the ordered
// target statistic is evaluated exactly as written, which makes it bit-exact
// against the GPU for binary labels.
//
// Steps and the passages they follow:
//   permutation      Section 2, the random permutation sigma before Eq. 1
//                    (generator: SplitMix64, Steele, Lea & Flood 2014; a reading,
//                    the paper names none)
//   prior            Section 2, the prior P after Eq. 1
//   ordered TS       Section 2, Eq. 1
//   borders / bins   Section 5 "Dense numerical features" (fixed number of bins,
//                    at most 255 per feature, 8 bits per feature)
//   gradients        Section 3, g = dLoss/da, Algorithm 1
//   histogram        Section 5, hist[j][b] = sum over rows with f_j = b of g
//   split score      Section 3 (enumerate splits, set leaf values, score the
//                    tree) + Section 4 "Fast scorer" (one split per level)
//   leaf index       Section 4 "Fast scorer": leaf = sum_i 2^i B(x, f(t,i))
//   leaf values      Section 3: gradient / Newton step leaf values
//   full-data TS     Section 2 (Eq. 1 with every training row "before" a new row):
//                    the statistic of a row that is not in the training permutation
//   prediction       Section 4 "Fast scorer": a row's model value is the sum over
//                    trees of the value of the leaf its binary features select
//   ordered boosting Section 3 "Fighting Gradient Bias", Algorithm 1 with the
//                    log-scale supporting models M'_i and shared tree structures
//   combinations     Section 2 "Feature combinations": greedy categorical feature
//                    combinations, converted to numbers by Eq. 1 on the fly
//
// Parity pins for every function live in tests/test_oracle_*.py.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <utility>
#include <set>
#include <vector>

namespace {

constexpr int LOSS_RMSE = 0;
constexpr int LOSS_LOGLOSS = 1;
constexpr int DTYPE_F32 = 0;
constexpr int DTYPE_BF16 = 1;
constexpr int LABEL_BINARY = 0;

// SplitMix64: output i of the generator seeded with `seed` is mix(seed + (i+1)*gamma).
uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ULL;
  uint64_t z = seed + (i + 1) * gamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Round a float to bfloat16 (round to nearest, ties to even) and back.
float round_to_bf16(float v) {
  if (std::isnan(v)) return v;
  uint32_t u;
  std::memcpy(&u, &v, 4);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// The value a gradient takes once it is stored: first rounded to FP32, then
// (for BF16 storage) to bfloat16.
double stored(double v, int dtype) {
  float f = static_cast<float>(v);
  if (dtype == DTYPE_BF16) f = round_to_bf16(f);
  return static_cast<double>(f);
}

double score_term(double G, double H, double l2) {
  double den = H + l2;
  if (den == 0.0) return 0.0;
  return G * G / den;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- permutation
uint64_t or_splitmix64(uint64_t seed, uint64_t i) { return splitmix64_at(seed, i); }

// sigma = row indices ordered by (key_i, i), key_i = SplitMix64 output i.
void or_make_permutation(uint64_t seed, int64_t n, uint32_t* perm) {
  std::vector<std::pair<uint64_t, uint32_t>> kv(n);
  for (int64_t i = 0; i < n; ++i) kv[i] = {splitmix64_at(seed, i), static_cast<uint32_t>(i)};
  std::sort(kv.begin(), kv.end());
  for (int64_t p = 0; p < n; ++p) perm[p] = kv[p].second;
}

// ---------------------------------------------------------------------- prior
// Binary labels: fraction of positive rows. Real labels: mean label, summed in
// row order.
double or_prior(const float* y, int64_t n, int label_kind) {
  if (label_kind == LABEL_BINARY) {
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) pos += (y[i] == 1.0f) ? 1 : 0;
    return static_cast<double>(pos) / static_cast<double>(n);
  }
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += static_cast<double>(y[i]);
  return s / static_cast<double>(n);
}

// ----------------------------------------------------------------- ordered TS
// Eq. 1 for one categorical column: walk the rows in permutation order keeping,
// per category, the label sum S and count N of the rows already seen; the row at
// position p gets (S + a*P) / (N + a) before its own label is added.
// cnt_before / sum_before (optional) receive N and S per row (row order).
void or_ordered_ts(const uint32_t* cat, const float* y, int64_t n, const uint32_t* perm,
                   double prior, double a, float* ts, uint32_t* cnt_before, double* sum_before) {
  std::unordered_map<uint32_t, std::pair<double, uint64_t>> seen;
  seen.reserve(static_cast<size_t>(n < 1024 ? 1024 : n / 4));
  for (int64_t p = 0; p < n; ++p) {
    uint32_t r = perm[p];
    auto& st = seen[cat[r]];
    double num = st.first + a * prior;
    double den = static_cast<double>(st.second) + a;
    ts[r] = static_cast<float>(num / den);
    if (cnt_before) cnt_before[r] = static_cast<uint32_t>(st.second);
    if (sum_before) sum_before[r] = st.first;
    st.first += static_cast<double>(y[r]);
    st.second += 1;
  }
}

// Literal O(n^2) evaluation of Eq. 1 (numerator and denominator summed over
// j < p), for tiny inputs only.
void or_ordered_ts_quadratic(const uint32_t* cat, const float* y, int64_t n, const uint32_t* perm,
                             double prior, double a, float* ts) {
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < p; ++j) {
      if (cat[perm[j]] == cat[perm[p]]) {
        s += static_cast<double>(y[perm[j]]);
        c += 1.0;
      }
    }
    ts[perm[p]] = static_cast<float>((s + a * prior) / (c + a));
  }
}

// -------------------------------------------------------------------- borders
// Borders of one column: v = the column sorted ascending; candidate k (1..B) is
// v[floor(k*n/(B+1))]; keep the strictly increasing values below max(v). A -0.0
// border is stored as +0.0. Returns the number of borders, or -1 if the column
// holds a NaN or an infinity.
int or_select_borders(const float* x, int64_t n, int max_borders, float* borders) {
  std::vector<float> v(x, x + n);
  for (float f : v)
    if (!std::isfinite(f)) return -1;
  std::sort(v.begin(), v.end());
  const float vmax = v[n - 1];
  int count = 0;
  for (int k = 1; k <= max_borders; ++k) {
    int64_t idx = (static_cast<int64_t>(k) * n) / (max_borders + 1);
    float c = v[idx];
    if (c == 0.0f) c = 0.0f;  // canonical +0
    if (!(c < vmax)) continue;
    if (count > 0 && !(c > borders[count - 1])) continue;
    borders[count++] = c;
  }
  return count;
}

// ------------------------------------------------------------------- quantise
// bin = number of borders strictly below x. x is column-major [F][n]; bins is
// row-major [n][F_pad] and feature f goes to column f_offset + f. When `rows`
// is given only those m rows are written (sampling at large sizes).
void or_quantize(const float* x, int64_t n, int F, const float* borders, const int* n_borders,
                 int max_borders, uint8_t* bins, int F_pad, int f_offset, const int64_t* rows,
                 int64_t m) {
  int64_t count = rows ? m : n;
  for (int64_t t = 0; t < count; ++t) {
    int64_t r = rows ? rows[t] : t;
    for (int f = 0; f < F; ++f) {
      const float* b = borders + static_cast<int64_t>(f) * max_borders;
      float v = x[static_cast<int64_t>(f) * n + r];
      int bin = static_cast<int>(std::lower_bound(b, b + n_borders[f], v) - b);
      bins[r * F_pad + f_offset + f] = static_cast<uint8_t>(bin);
    }
  }
}

// ------------------------------------------------------------------ gradients
// RMSE: g = pred - y, h = 1. Logloss: p = 1/(1+exp(-pred)), g = p - y,
// h = p(1-p). Both are then rounded to the storage type.
void or_gradients(int loss, const float* y, const double* pred, int64_t n, int dtype, double* g,
                  double* h) {
  for (int64_t i = 0; i < n; ++i) {
    double gi, hi;
    if (loss == LOSS_RMSE) {
      gi = pred[i] - static_cast<double>(y[i]);
      hi = 1.0;
    } else {
      double p = 1.0 / (1.0 + std::exp(-pred[i]));
      gi = p - static_cast<double>(y[i]);
      hi = p * (1.0 - p);
    }
    g[i] = stored(gi, dtype);
    h[i] = stored(hi, dtype);
  }
}

double or_round_bf16(double v) { return static_cast<double>(round_to_bf16(static_cast<float>(v))); }

// ------------------------------------------------------------------ histogram
// hist[l][f][b][s] = sum over rows r with leaf[r] = l and bins[r][f] = b of
// (g_r, h_r)[s], summed in row order. Layout [L][F][max_bins][2].
void or_histogram(const uint8_t* bins, int64_t n, int F_pad, int F, const double* g,
                  const double* h, const uint16_t* leaf, int n_leaves, int max_bins,
                  double* hist) {
  std::fill(hist, hist + static_cast<int64_t>(n_leaves) * F * max_bins * 2, 0.0);
  for (int64_t r = 0; r < n; ++r) {
    int l = leaf ? leaf[r] : 0;
    for (int f = 0; f < F; ++f) {
      int b = bins[r * F_pad + f];
      double* cell = hist + ((static_cast<int64_t>(l) * F + f) * max_bins + b) * 2;
      cell[0] += g[r];
      cell[1] += h[r];
    }
  }
}

// -------------------------------------------------------------- split scores
// For every feature f with n_borders[f] > 0 and border k < n_borders[f]:
//   score(f,k) = sum over leaves l of  G_L^2/(H_L+l2) + G_R^2/(H_R+l2)
// with L = bins <= k and R = bins > k of leaf l; a term whose denominator is 0
// counts as 0. scores is [F][max_bins-1]; invalid candidates get -inf.
// The best candidate is the largest score, exact ties going to the smallest f,
// then the smallest k; second receives the second-largest score over all
// candidates. Returns 0, or -1 if there is no candidate at all.
int or_split_scores(const double* hist, int n_leaves, int F, const int* n_borders, int max_bins,
                    double l2, double* scores, int* best_f, int* best_k, double* best_score,
                    double* second_score) {
  const int K = max_bins - 1;
  const double ninf = -INFINITY;
  std::vector<double> sufG(max_bins + 1), sufH(max_bins + 1);
  for (int f = 0; f < F; ++f) {
    double* sf = scores + static_cast<int64_t>(f) * K;
    for (int k = 0; k < K; ++k) sf[k] = (k < n_borders[f]) ? 0.0 : ninf;
    if (n_borders[f] <= 0) continue;
    for (int l = 0; l < n_leaves; ++l) {
      const double* hl = hist + (static_cast<int64_t>(l) * F + f) * max_bins * 2;
      // running sums over bins above k, from the top
      sufG[max_bins] = 0.0;
      sufH[max_bins] = 0.0;
      for (int b = max_bins - 1; b >= 0; --b) {
        sufG[b] = sufG[b + 1] + hl[2 * b];
        sufH[b] = sufH[b + 1] + hl[2 * b + 1];
      }
      double GL = 0.0, HL = 0.0;
      for (int k = 0; k < n_borders[f]; ++k) {
        GL += hl[2 * k];
        HL += hl[2 * k + 1];
        sf[k] += score_term(GL, HL, l2) + score_term(sufG[k + 1], sufH[k + 1], l2);
      }
    }
  }
  int bf = -1, bk = -1;
  double bs = ninf, ss = ninf;
  for (int f = 0; f < F; ++f) {
    for (int k = 0; k < n_borders[f] && k < K; ++k) {
      double s = scores[static_cast<int64_t>(f) * K + k];
      if (bf < 0 || s > bs) {
        if (bf >= 0) ss = std::max(ss, bs);
        bs = s;
        bf = f;
        bk = k;
      } else {
        ss = std::max(ss, s);
      }
    }
  }
  *best_f = bf;
  *best_k = bk;
  *best_score = bs;
  *second_score = ss;
  return bf < 0 ? -1 : 0;
}

// ----------------------------------------------------------------- leaf index
// Level d of an oblivious tree: leaf[r] += 2^d * [bins[r][f] > k].
void or_update_leaf(const uint8_t* bins, int64_t n, int F_pad, int f, int k, int d,
                    uint16_t* leaf) {
  if (f < 0) return;
  for (int64_t r = 0; r < n; ++r)
    if (bins[r * F_pad + f] > k) leaf[r] = static_cast<uint16_t>(leaf[r] + (1u << d));
}

// Leaf index of every row for a whole tree (the scorer's encoding):
// leaf = sum_i 2^i * [bins[r][f_i] > k_i]; levels with f_i < 0 add nothing.
void or_tree_leaf_index(const uint8_t* bins, int64_t n, int F_pad, const int* f, const int* k,
                        int depth, uint16_t* leaf) {
  for (int64_t r = 0; r < n; ++r) {
    unsigned idx = 0;
    for (int i = 0; i < depth; ++i)
      if (f[i] >= 0 && bins[r * F_pad + f[i]] > k[i]) idx += 1u << i;
    leaf[r] = static_cast<uint16_t>(idx);
  }
}

// --------------------------------------------------------------- leaf values
// Per-leaf totals (G, H) summed in row order, then the Newton step
// v = -G/(H + l2) (0 when the denominator is 0).
void or_leaf_totals(const double* g, const double* h, const uint16_t* leaf, int64_t n,
                    int n_leaves, double* tot) {
  std::fill(tot, tot + 2 * n_leaves, 0.0);
  for (int64_t r = 0; r < n; ++r) {
    tot[2 * leaf[r]] += g[r];
    tot[2 * leaf[r] + 1] += h[r];
  }
}

void or_leaf_values(const double* tot, int n_leaves, double l2, double* v) {
  for (int l = 0; l < n_leaves; ++l) {
    double den = tot[2 * l + 1] + l2;
    v[l] = (den == 0.0) ? 0.0 : -tot[2 * l] / den;
  }
}

void or_apply_leaf_values(const uint16_t* leaf, int64_t n, const double* v, double lr,
                          double* pred) {
  for (int64_t r = 0; r < n; ++r) pred[r] += lr * v[leaf[r]];
}

// ----------------------------------------------------------------------- loss
double or_loss(int loss, const float* y, const double* pred, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double yi = static_cast<double>(y[i]);
    if (loss == LOSS_RMSE) {
      double e = yi - pred[i];
      s += e * e;
    } else {
      double p = 1.0 / (1.0 + std::exp(-pred[i]));
      s += -(yi * std::log(p) + (1.0 - yi) * std::log(1.0 - p));
    }
  }
  s /= static_cast<double>(n);
  return loss == LOSS_RMSE ? std::sqrt(s) : s;
}

// ------------------------------------------------------------------ lock step
// Where the best and the runner-up split differ by at most a rounding-sized margin, the
// paper's greedy search (Section 3, one split per level, Section 4 "Fast scorer") does not
// fix the choice: an implementation that accumulates in another order may take either.
// To follow such an implementation through a whole run, the oracle can be given its
// split for every level ("follow"). At a level where the followed split (ff, fk) is not
// the oracle's own best, the oracle takes it if its score here is within
// tol * |best| of the best (a near-tie: flag 1) and keeps its own otherwise (flag -1:
// a genuine disagreement, which a test reports). Flag 0: the two agree. Only the choice
// changes; every score, total and leaf value is computed exactly as without a follow.
static int follow_split(const double* scores, int F, int K, const int* n_borders, int ff, int fk, double tol,
                        int* bf, int* bk, double bs) {
  if (ff == *bf && fk == *bk) return 0;
  if (ff < 0 || ff >= F || fk < 0 || fk >= n_borders[ff] || fk >= K) return -1;
  const double sf = scores[static_cast<int64_t>(ff) * K + fk];
  if (!(bs - sf <= tol * std::fabs(bs))) return -1;
  *bf = ff;
  *bk = fk;
  return 1;
}

// ------------------------------------------------------------------- boosting
// Classic (non-ordered) boosting of T oblivious trees of depth D on quantised
// features, starting from pred = 0 (pred is in/out, FP64). Per tree: gradients
// (rounded to the storage type), D levels of histogram + best split + leaf
// update, then Newton leaf values and pred += lr * v[leaf].
// Outputs per tree t and level d (arrays [T][D]): chosen feature and border,
// best and second-best score; per tree: leaf values v [T][2^D] (before lr) and
// the training loss after the tree [T].
// follow_f / follow_k (optional, [T][D]): another implementation's splits, taken at
// near-ties within follow_tol (see follow_split); followed [T][D] receives the flags.
void or_fit(const uint8_t* bins, int64_t n, int F_pad, int F, const int* n_borders, int max_bins,
            const float* y, int loss, int dtype, int depth, int trees, double lr, double l2,
            double* pred, int* split_f, int* split_k, double* split_score, double* split_second,
            double* leaf_values, double* losses, const int* follow_f, const int* follow_k, double follow_tol,
            int* followed) {
  const int L = 1 << depth;
  std::vector<double> g(n), h(n);
  std::vector<uint16_t> leaf(n);
  std::vector<double> hist(static_cast<size_t>(L / 2 > 0 ? L / 2 : 1) * F * max_bins * 2);
  std::vector<double> scores(static_cast<size_t>(F) * (max_bins > 1 ? max_bins - 1 : 1));
  std::vector<double> tot(2 * L), v(L);
  for (int t = 0; t < trees; ++t) {
    or_gradients(loss, y, pred, n, dtype, g.data(), h.data());
    std::fill(leaf.begin(), leaf.end(), 0);
    for (int d = 0; d < depth; ++d) {
      int nl = 1 << d;
      or_histogram(bins, n, F_pad, F, g.data(), h.data(), leaf.data(), nl, max_bins, hist.data());
      int bf, bk;
      double bs, ss;
      or_split_scores(hist.data(), nl, F, n_borders, max_bins, l2, scores.data(), &bf, &bk, &bs,
                      &ss);
      if (follow_f && bf >= 0)
        followed[t * depth + d] = follow_split(scores.data(), F, max_bins > 1 ? max_bins - 1 : 1, n_borders,
                                               follow_f[t * depth + d], follow_k[t * depth + d], follow_tol, &bf,
                                               &bk, bs);
      else if (follow_f)
        followed[t * depth + d] = follow_f[t * depth + d] == bf ? 0 : -1;
      split_f[t * depth + d] = bf;
      split_k[t * depth + d] = bk;
      split_score[t * depth + d] = bs;
      split_second[t * depth + d] = ss;
      or_update_leaf(bins, n, F_pad, bf, bk, d, leaf.data());
    }
    or_leaf_totals(g.data(), h.data(), leaf.data(), n, L, tot.data());
    or_leaf_values(tot.data(), L, l2, v.data());
    for (int l = 0; l < L; ++l) leaf_values[static_cast<int64_t>(t) * L + l] = v[l];
    or_apply_leaf_values(leaf.data(), n, v.data(), lr, pred);
    losses[t] = or_loss(loss, y, pred, n);
  }
}

// ------------------------------------------------------------- full-data TS
// For rows outside the training data (inference), every training row counts as
// "before": per category, S = sum of the labels and N = the number of training rows
// with that category (in row order); a new row with category c gets
// (S_c + a*P) / (N_c + a), and an unseen category gets (0 + a*P) / (0 + a).
void or_ts_full(const uint32_t* cat, const float* y, int64_t n, double prior, double a,
                const uint32_t* cat_new, int64_t m, float* ts) {
  std::unordered_map<uint32_t, std::pair<double, double>> stats;
  for (int64_t r = 0; r < n; ++r) {
    auto& st = stats[cat[r]];
    st.first += static_cast<double>(y[r]);
    st.second += 1.0;
  }
  for (int64_t i = 0; i < m; ++i) {
    auto it = stats.find(cat_new[i]);
    const double S = it == stats.end() ? 0.0 : it->second.first;
    const double N = it == stats.end() ? 0.0 : it->second.second;
    ts[i] = static_cast<float>((S + a * prior) / (N + a));
  }
}

// --------------------------------------------------------------- prediction
// Model value of every row: sum over trees t (in order) of lr * v_t[leaf_t(row)],
// where leaf_t(row) = sum_d 2^d [bin(row, f_td) > k_td] (a level with f_td < 0 sends
// every row to its 0 side). bins is row-major [n][F_pad]; split_f, split_k are
// [T][D] and leaf_values [T][2^D] (before the learning rate).
void or_predict(const uint8_t* bins, int64_t n, int F_pad, const int* split_f, const int* split_k,
                const double* leaf_values, int trees, int depth, double lr, double* pred) {
  const int64_t L = int64_t(1) << depth;
  for (int64_t r = 0; r < n; ++r) {
    double s = 0.0;
    for (int t = 0; t < trees; ++t) {
      int64_t leaf = 0;
      for (int d = 0; d < depth; ++d) {
        const int f = split_f[t * depth + d];
        if (f >= 0 && bins[r * F_pad + f] > split_k[t * depth + d]) leaf |= int64_t(1) << d;
      }
      s += lr * leaf_values[t * L + leaf];
    }
    pred[r] = s;
  }
}

// ---------------------------------------------------------- ordered boosting
// Ordered boosting (Section 3, Algorithm 1) in the log-scale form the section describes,
// with these readings where it is silent:
//  - s permutations sigma_q (perms [s][n], position -> row). Each has its own bins
//    (bins [s][n][F_pad], row order): the float columns are shared, the categorical
//    columns hold the ordered TS computed along sigma_q (the section uses the TS
//    permutations for the gradients too), quantised with one set of borders;
//  - tree t takes its structure from permutation r = t mod s: bins of sigma_r and the
//    ordered gradients of sigma_r;
//  - positions are 0-based. The supporting model M'_{q,i}, i = 0..floor(log2(n-1)), is
//    trained on positions p < 2^i of sigma_q and holds values for positions
//    j < min(2^(i+1), n). The gradient at position k >= 1 is taken at
//    M'_{r, floor(log2 k)}(x_k), trained on positions < 2^floor(log2 k) <= k, so never
//    on x_k itself; position 0 has no earlier sample and takes the starting value 0;
//  - the structure is searched greedily level by level on those gradients exactly as in
//    classic boosting (histograms, score, leaf update);
//  - the final model's leaf values are Newton steps on the plain gradients of all rows
//    at its own prediction (the second phase, done the classic way), with leaf indices
//    on the bins of permutation 0;
//  - every supporting model of every permutation takes the same structure (leaf indices
//    on its permutation's bins) and Newton leaf values from the gradients at its own
//    values on its first 2^i positions, added (times lr) at all positions it holds.
// Gradients are rounded to FP32 storage as in or_fit. sup_out (optional) receives the
// supporting values [s][n_sup], n_sup = sum_i min(2^(i+1), n), models in order of i,
// each model's values by position. follow_f / follow_k / follow_tol / followed: the lock
// step of or_fit (follow_split).
static int floor_log2(int64_t k) {
  int r = 0;
  while ((int64_t(1) << (r + 1)) <= k) ++r;
  return r;
}

int64_t or_ordered_sup_size(int64_t n) {
  if (n <= 0) return 0;
  const int I = n > 1 ? floor_log2(n - 1) : 0;
  int64_t tot = 0;
  for (int i = 0; i <= I; ++i) tot += std::min<int64_t>(int64_t(2) << i, n);
  return tot;
}

void or_fit_ordered(const uint8_t* bins, int64_t n, int F_pad, int F, const int* n_borders, int max_bins,
                    const float* y, int loss, int depth, int trees, double lr, double l2, const uint32_t* perms,
                    int s, double* pred, int* split_f, int* split_k, double* split_score, double* split_second,
                    double* leaf_values, double* losses, double* sup_out, const int* follow_f,
                    const int* follow_k, double follow_tol, int* followed) {
  const int L = 1 << depth;
  const int I = n > 1 ? floor_log2(n - 1) : 0;
  std::vector<int64_t> off(I + 2, 0);
  for (int i = 0; i <= I; ++i) off[i + 1] = off[i] + std::min<int64_t>(int64_t(2) << i, n);
  const int64_t n_sup = off[I + 1];
  const size_t plane = static_cast<size_t>(n) * F_pad;
  std::vector<double> sup(static_cast<size_t>(s) * n_sup, 0.0);
  std::vector<double> go(n), ho(n), gp(n), hp(n);
  std::vector<uint16_t> leaf(n), leafq(n);
  std::vector<double> hist(static_cast<size_t>(L / 2 > 0 ? L / 2 : 1) * F * max_bins * 2);
  std::vector<double> scores(static_cast<size_t>(F) * (max_bins > 1 ? max_bins - 1 : 1));
  std::vector<double> tot(2 * L), v(L);
  auto grad = [&](double a, float yv, double* g, double* h) { or_gradients(loss, &yv, &a, 1, 0, g, h); };
  for (int t = 0; t < trees; ++t) {
    const int r = t % s;
    const uint32_t* sig = perms + static_cast<int64_t>(r) * n;
    const uint8_t* bins_r = bins + r * plane;
    const double* sup_r = sup.data() + static_cast<size_t>(r) * n_sup;
    // gradients for the structure: position k from M'_{r, floor(log2 k)}
    for (int64_t k = 0; k < n; ++k) {
      const double a = k == 0 ? 0.0 : sup_r[off[floor_log2(k)] + k];
      grad(a, y[sig[k]], &go[sig[k]], &ho[sig[k]]);
    }
    std::fill(leaf.begin(), leaf.end(), 0);
    for (int d = 0; d < depth; ++d) {
      int bf, bk;
      double bs, ss;
      or_histogram(bins_r, n, F_pad, F, go.data(), ho.data(), leaf.data(), 1 << d, max_bins, hist.data());
      or_split_scores(hist.data(), 1 << d, F, n_borders, max_bins, l2, scores.data(), &bf, &bk, &bs, &ss);
      if (follow_f && bf >= 0)
        followed[t * depth + d] = follow_split(scores.data(), F, max_bins > 1 ? max_bins - 1 : 1, n_borders,
                                               follow_f[t * depth + d], follow_k[t * depth + d], follow_tol, &bf,
                                               &bk, bs);
      else if (follow_f)
        followed[t * depth + d] = follow_f[t * depth + d] == bf ? 0 : -1;
      split_f[t * depth + d] = bf;
      split_k[t * depth + d] = bk;
      split_score[t * depth + d] = bs;
      split_second[t * depth + d] = ss;
      or_update_leaf(bins_r, n, F_pad, bf, bk, d, leaf.data());
    }
    const int* tf = split_f + t * depth;
    const int* tk = split_k + t * depth;
    // the final model: plain gradients of every row at its prediction
    or_tree_leaf_index(bins, n, F_pad, tf, tk, depth, leafq.data());
    or_gradients(loss, y, pred, n, 0, gp.data(), hp.data());
    or_leaf_totals(gp.data(), hp.data(), leafq.data(), n, L, tot.data());
    or_leaf_values(tot.data(), L, l2, v.data());
    for (int l = 0; l < L; ++l) leaf_values[static_cast<int64_t>(t) * L + l] = v[l];
    or_apply_leaf_values(leafq.data(), n, v.data(), lr, pred);
    losses[t] = or_loss(loss, y, pred, n);
    // the supporting models of every permutation
    for (int q = 0; q < s; ++q) {
      const uint32_t* sq = perms + static_cast<int64_t>(q) * n;
      or_tree_leaf_index(bins + q * plane, n, F_pad, tf, tk, depth, leafq.data());
      double* sm = sup.data() + static_cast<size_t>(q) * n_sup;
      for (int i = 0; i <= I; ++i) {
        const int64_t train = std::min<int64_t>(int64_t(1) << i, n);
        const int64_t held = std::min<int64_t>(int64_t(2) << i, n);
        std::fill(tot.begin(), tot.end(), 0.0);
        for (int64_t p = 0; p < train; ++p) {
          double g, h;
          grad(sm[off[i] + p], y[sq[p]], &g, &h);
          tot[2 * leafq[sq[p]]] += g;
          tot[2 * leafq[sq[p]] + 1] += h;
        }
        or_leaf_values(tot.data(), L, l2, v.data());
        for (int64_t j = 0; j < held; ++j) sm[off[i] + j] += lr * v[leafq[sq[j]]];
      }
    }
  }
  if (sup_out) std::copy(sup.begin(), sup.end(), sup_out);
}

// ----------------------------------------------------- feature combinations
// Section 2 "Feature combinations" with these readings where it is silent:
//  - an item is a categorical column c (its ids) or a split (f, k) already in the tree,
//    taken as a two-valued categorical feature [bin of f > k]; a combination is a set of
//    items, kept sorted by (kind, a, b) with categorical columns first;
//  - the value of a combination in a row is a SplitMix64 chain over its items in that
//    order, h <- splitmix64_at(h, v) from h = 0 (v = the id, or the bit), folded to 32
//    bits as h ^ (h >> 32); it is converted to a number by Eq. 1 along sigma (the same
//    prior and a as single columns), and quantised with borders chosen on that column;
//  - the first level of a tree takes no combinations. At level d >= 1 the items present
//    in the tree are: for every split so far, the set {c} for a split on the TS column of
//    categorical c, the set {(f, k)} for a split on a float feature, and the combination
//    itself for a combination split. Candidates are every present set joined with every
//    categorical column it lacks, up to max_complexity items, without repeats, in
//    lexicographic order of their sorted items;
//  - a candidate's best border is scored on the current leaves exactly as an ordinary
//    feature; it replaces the ordinary split only with a strictly higher score (ties to the
//    ordinary split, then to the first candidate, then the smallest border). A chosen
//    combination is recorded as feature F + j (j-th combination of the tree) and is not
//    scored again as an ordinary feature.
namespace {
struct ComboItem {
  int kind, a, b;   // kind 0: categorical column a (b = 0); kind 1: [bin of feature a > b]
  bool operator<(const ComboItem& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (a != o.a) return a < o.a;
    return b < o.b;
  }
  bool operator==(const ComboItem& o) const { return kind == o.kind && a == o.a && b == o.b; }
};
}  // namespace

// Ids of a combination for every row. items: [m][3] (kind, a, b) in canonical order.
void or_combo_ids(const int* items, int m, const uint32_t* cat, int64_t n, const uint8_t* bins, int F_pad,
                  uint32_t* ids) {
  for (int64_t r = 0; r < n; ++r) {
    uint64_t h = 0;
    for (int i = 0; i < m; ++i) {
      const int kind = items[3 * i], a = items[3 * i + 1], b = items[3 * i + 2];
      const uint64_t v = kind == 0 ? cat[static_cast<int64_t>(a) * n + r] : (bins[r * F_pad + a] > b ? 1u : 0u);
      h = splitmix64_at(h, v);
    }
    ids[r] = static_cast<uint32_t>(h ^ (h >> 32));
  }
}

void or_fit_combos(const uint8_t* bins, int64_t n, int F_pad, int F, int F_float, const int* n_borders, int max_bins,
                   const uint32_t* cat, const float* y, int loss, int depth, int trees, double lr, double l2,
                   const uint32_t* perm, double prior, double a, int max_borders, int max_complexity, double* pred,
                   int* split_f, int* split_k, double* split_score, double* split_second, double* leaf_values,
                   double* losses, int* combo_items, int* combo_nb, float* combo_borders) {
  const int L = 1 << depth;
  const int C = F - F_float;
  const int cmb = max_borders + 1;
  std::vector<double> g(n), h(n);
  std::vector<uint16_t> leaf(n);
  std::vector<double> hist(static_cast<size_t>(L / 2 > 0 ? L / 2 : 1) * F * max_bins * 2);
  std::vector<double> scores(static_cast<size_t>(F) * (max_bins > 1 ? max_bins - 1 : 1));
  std::vector<double> chist(static_cast<size_t>(L / 2 > 0 ? L / 2 : 1) * cmb * 2), cscores(cmb);
  std::vector<double> tot(2 * L), v(L);
  std::vector<uint32_t> ids(n);
  std::vector<float> ts(n), cb(max_borders > 0 ? max_borders : 1), best_b(cb.size());
  std::vector<uint8_t> colbins(static_cast<size_t>(n) * 32, 0), best_bins(static_cast<size_t>(n) * 32, 0);
  std::vector<int> flat;
  for (int t = 0; t < trees; ++t) {
    or_gradients(loss, y, pred, n, 0, g.data(), h.data());
    std::fill(leaf.begin(), leaf.end(), 0);
    std::vector<std::vector<ComboItem>> present;
    int n_combo = 0;
    for (int d = 0; d < depth; ++d) {
      const int64_t rec = static_cast<int64_t>(t) * depth + d;
      for (int i = 0; i < 3 * max_complexity; ++i) combo_items[rec * 3 * max_complexity + i] = -1;
      combo_nb[rec] = 0;
      for (int i = 0; i < max_borders; ++i) combo_borders[rec * max_borders + i] = 0.0f;
      const int nl = 1 << d;
      int bf, bk;
      double bs, ss;
      or_histogram(bins, n, F_pad, F, g.data(), h.data(), leaf.data(), nl, max_bins, hist.data());
      or_split_scores(hist.data(), nl, F, n_borders, max_bins, l2, scores.data(), &bf, &bk, &bs, &ss);
      double top1 = -INFINITY, top2 = -INFINITY;
      auto push = [&](double sc) {
        if (sc > top1) {
          top2 = top1;
          top1 = sc;
        } else if (sc > top2) {
          top2 = sc;
        }
      };
      if (bf >= 0) {
        push(bs);
        push(ss);
      }
      // candidates
      std::set<std::vector<ComboItem>> cands;
      if (d >= 1)
        for (const auto& p : present)
          for (int c = 0; c < C; ++c) {
            const ComboItem it{0, c, 0};
            if (std::find(p.begin(), p.end(), it) != p.end() || static_cast<int>(p.size()) + 1 > max_complexity)
              continue;
            std::vector<ComboItem> q = p;
            q.push_back(it);
            std::sort(q.begin(), q.end());
            cands.insert(q);
          }
      const std::vector<ComboItem>* win = nullptr;
      int wk = -1, wnb = 0;
      double ws = -INFINITY;
      for (const auto& q : cands) {
        flat.clear();
        for (const auto& it : q) flat.insert(flat.end(), {it.kind, it.a, it.b});
        or_combo_ids(flat.data(), static_cast<int>(q.size()), cat, n, bins, F_pad, ids.data());
        or_ordered_ts(ids.data(), y, n, perm, prior, a, ts.data(), nullptr, nullptr);
        const int nb = or_select_borders(ts.data(), n, max_borders, cb.data());
        if (nb <= 0) continue;
        or_quantize(ts.data(), n, 1, cb.data(), &nb, max_borders, colbins.data(), 32, 0, nullptr, 0);
        int cf, ck;
        double cs, css;
        or_histogram(colbins.data(), n, 32, 1, g.data(), h.data(), leaf.data(), nl, cmb, chist.data());
        or_split_scores(chist.data(), nl, 1, &nb, cmb, l2, cscores.data(), &cf, &ck, &cs, &css);
        if (cf < 0) continue;
        push(cs);
        push(css);
        if (!win || cs > ws) {
          win = &q;
          wk = ck;
          ws = cs;
          wnb = nb;
          best_bins.swap(colbins);
          std::copy(cb.begin(), cb.end(), best_b.begin());
        }
      }
      split_score[rec] = top1;
      split_second[rec] = top2;
      if (win && (bf < 0 || ws > bs)) {
        split_f[rec] = F + n_combo;
        split_k[rec] = wk;
        for (size_t i = 0; i < win->size(); ++i) {
          combo_items[(rec * max_complexity + i) * 3] = (*win)[i].kind;
          combo_items[(rec * max_complexity + i) * 3 + 1] = (*win)[i].a;
          combo_items[(rec * max_complexity + i) * 3 + 2] = (*win)[i].b;
        }
        combo_nb[rec] = wnb;
        for (int i = 0; i < wnb; ++i) combo_borders[rec * max_borders + i] = best_b[i];
        or_update_leaf(best_bins.data(), n, 32, 0, wk, d, leaf.data());
        if (std::find(present.begin(), present.end(), *win) == present.end()) present.push_back(*win);
        ++n_combo;
      } else {
        split_f[rec] = bf;
        split_k[rec] = bk;
        or_update_leaf(bins, n, F_pad, bf, bk, d, leaf.data());
        if (bf >= 0) {
          const std::vector<ComboItem> p{bf < F_float ? ComboItem{1, bf, bk} : ComboItem{0, bf - F_float, 0}};
          if (std::find(present.begin(), present.end(), p) == present.end()) present.push_back(p);
        }
      }
    }
    or_leaf_totals(g.data(), h.data(), leaf.data(), n, L, tot.data());
    or_leaf_values(tot.data(), L, l2, v.data());
    for (int l = 0; l < L; ++l) leaf_values[static_cast<int64_t>(t) * L + l] = v[l];
    or_apply_leaf_values(leaf.data(), n, v.data(), lr, pred);
    losses[t] = or_loss(loss, y, pred, n);
  }
}

}  // extern "C"
