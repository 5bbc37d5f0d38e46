// symbolic.cpp -- host symbolic phase of the block ILU(k) library.
//
// Section 2.3: the block matrix is abstracted to its block graph (every listed
// block is one point, whatever its values).  Section 2.2, Algorithm 3 with
// Eq. 1 and Eq. 2 gives the level-of-fill pattern P'; Section 2.4, Eq. 4 gives
// the dependency levels of the two triangular solves.  Everything here depends
// on the pattern only, never on values, which is what lets the factorization
// reuse it (the decoupling argument of Section 1).
//
// Row i is built by a pivot-driven merge: a min-heap releases the pivots
// p < i of row i in ascending column order (each pivot's level is final when it
// leaves the heap, because only smaller pivots can lower it), and every pivot
// of level <= k offers lev_ip + lev_pj + 1 to the columns j > p of P'(p)
// (Eq. 2).  Candidates above k are discarded at once: a level only decreases,
// so such a candidate could never survive the final lev <= k test.

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <queue>
#include <vector>

#include "bilu_internal.h"

namespace {

int check_pattern(int32_t n, const int32_t* rp, const int32_t* ci) {
  if (n < 0) return BILU_ERR_ARG;
  if (n == 0) return BILU_OK;
  if (!rp || (rp[n] > 0 && !ci)) return BILU_ERR_ARG;
  if (rp[0] != 0) return BILU_ERR_PATTERN;
  for (int32_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return BILU_ERR_PATTERN;
    bool diag = false;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
      const int32_t j = ci[t];
      if (j < 0 || j >= n) return BILU_ERR_PATTERN;
      if (t > rp[i] && j <= ci[t - 1]) return BILU_ERR_PATTERN;
      diag |= (j == i);
    }
    if (!diag) return BILU_ERR_PATTERN;
  }
  return BILU_OK;
}

// Eq. 4 levels and the L / U' split of a pattern whose rp, ci (and n) are set.
void finish_pattern(bilu_pattern* p) {
  const int32_t n = p->n;
  // Eq. 4 on the lower part (rows ascending) and on the reversed graph of the
  // upper part (rows descending); 0-based.
  p->lvl_l.assign((size_t)n, 0);
  p->lvl_u.assign((size_t)n, 0);
  int32_t ml = -1, mu = -1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int32_t t = p->rp[i]; t < p->rp[i + 1] && p->ci[t] < i; ++t)
      l = std::max(l, p->lvl_l[p->ci[t]] + 1);
    p->lvl_l[i] = l;
    ml = std::max(ml, l);
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int32_t t = p->rp[i + 1] - 1; t >= p->rp[i] && p->ci[t] > i; --t)
      l = std::max(l, p->lvl_u[p->ci[t]] + 1);
    p->lvl_u[i] = l;
    mu = std::max(mu, l);
  }
  p->nlev_l = ml + 1;
  p->nlev_u = mu + 1;

  // Split P' into strictly lower and strictly upper CSR structures.
  p->max_l = p->max_u = p->line_len = 0;
  p->lrp.assign((size_t)n + 1, 0);
  p->urp.assign((size_t)n + 1, 0);
  for (int32_t i = 0; i < n; ++i) {
    int32_t nl = 0, nu = 0;
    for (int32_t t = p->rp[i]; t < p->rp[i + 1]; ++t) {
      if (p->ci[t] < i) ++nl;
      else if (p->ci[t] > i) ++nu;
    }
    p->lrp[(size_t)i + 1] = p->lrp[i] + nl;
    p->urp[(size_t)i + 1] = p->urp[i] + nu;
    p->max_l = std::max(p->max_l, nl);
    p->max_u = std::max(p->max_u, nu);
  }
  p->lci.resize((size_t)p->lrp[n]);
  p->uci.resize((size_t)p->urp[n]);
  p->cnt_p = (int64_t)p->ci.size();
  p->cnt_l = (int64_t)p->lci.size();
  p->cnt_u = (int64_t)p->uci.size();
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = p->lrp[i], c = p->urp[i];
    for (int32_t t = p->rp[i]; t < p->rp[i + 1]; ++t) {
      if (p->ci[t] < i) p->lci[a++] = p->ci[t];
      else if (p->ci[t] > i) p->uci[c++] = p->ci[t];
    }
  }

  // Line length: the most common distance (up to 4096) between consecutive
  // rows that do not depend on row i - 1.
  std::vector<int32_t> hist(4097, 0);
  int32_t prev = -1;
  for (int32_t i = 0; i < n; ++i) {
    const int32_t e = p->lrp[(size_t)i + 1];
    if (e > p->lrp[i] && p->lci[(size_t)e - 1] == i - 1) continue;  // depends on its predecessor
    if (prev >= 0 && i - prev <= 4096) ++hist[(size_t)(i - prev)];
    prev = i;
  }
  int32_t best = 0;
  for (int32_t d = 2; d <= 4096; ++d)
    if (hist[(size_t)d] > hist[(size_t)best] && hist[(size_t)d] >= 2) best = d;
  p->line_len = best;
}

}  // namespace

namespace bilu {

// Eq. 4 levels, the L / U' split and the backfill gather map (Algorithm 5
// steps 3-4: slot -> A block or -1) of a pattern whose n, k, nnz_a, rp, ci and
// lev are set (by the host symbolic phase or the device one).
int complete_pattern(bilu_pattern* p, const int32_t* row_ptr, const int32_t* col_idx) {
  const int32_t n = p->n;
  finish_pattern(p);
  const int64_t nl = p->nnz_l(), nslots = p->nslots();
  if (nslots > (int64_t)INT32_MAX) return BILU_ERR_OOM;
  p->slot_src.assign((size_t)nslots, -1);
  for (int32_t i = 0; i < n; ++i) {
    int32_t a = p->lrp[i], c = p->urp[i];
    for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
      const int32_t j = col_idx[t];
      int64_t slot;
      if (j < i) {
        while (p->lci[a] != j) ++a;  // A's pattern is a subset of P'
        slot = a;
      } else if (j == i) {
        slot = nl + i;
      } else {
        while (p->uci[c] != j) ++c;
        slot = nl + n + c;
      }
      p->slot_src[(size_t)slot] = t;
    }
  }
  return BILU_OK;
}

// The block CSR checks of bilu_symbolic (sorted, unique, in range, diagonal
// present), for the device symbolic phase.
int validate_pattern(int32_t n, const int32_t* row_ptr, const int32_t* col_idx) {
  return check_pattern(n, row_ptr, col_idx);
}

}  // namespace bilu

extern "C" int bilu_symbolic(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t k,
                             bilu_pattern** out) {
  if (!out || k < 0) return BILU_ERR_ARG;
  *out = nullptr;
  int st = check_pattern(n, row_ptr, col_idx);
  if (st != BILU_OK) return st;
  bilu_pattern* p = new (std::nothrow) bilu_pattern();
  if (!p) return BILU_ERR_OOM;
  try {
    p->n = n;
    p->k = k;
    p->nnz_a = n > 0 ? row_ptr[n] : 0;
    p->rp.assign((size_t)n + 1, 0);
    p->ci.reserve((size_t)p->nnz_a * 2 + 16);
    p->lev.reserve((size_t)p->nnz_a * 2 + 16);

    std::vector<int32_t> mark((size_t)n, -1);   // mark[j] == i: column j is in row i
    std::vector<int32_t> level((size_t)n, 0);   // level of column j in the current row
    std::vector<int32_t> cols;
    std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> pivots;

    for (int32_t i = 0; i < n; ++i) {
      cols.clear();
      for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {  // Eq. 1
        const int32_t j = col_idx[t];
        mark[j] = i;
        level[j] = 0;
        cols.push_back(j);
        if (j < i) pivots.push(j);
      }
      while (!pivots.empty()) {
        const int32_t piv = pivots.top();
        pivots.pop();
        const int64_t lp = level[piv];
        if (lp > k) continue;
        for (int32_t t = p->rp[piv]; t < p->rp[piv + 1]; ++t) {
          const int32_t j = p->ci[t];
          if (j <= piv) continue;
          const int64_t cand = lp + p->lev[t] + 1;  // Eq. 2
          if (cand > k) continue;
          if (mark[j] != i) {
            mark[j] = i;
            level[j] = (int32_t)cand;
            cols.push_back(j);
            if (j < i) pivots.push(j);
          } else if (cand < level[j]) {
            level[j] = (int32_t)cand;
          }
        }
      }
      std::sort(cols.begin(), cols.end());
      if ((int64_t)p->ci.size() + (int64_t)cols.size() > (int64_t)INT32_MAX) {
        delete p;
        return BILU_ERR_OOM;
      }
      for (int32_t j : cols) {
        p->ci.push_back(j);
        p->lev.push_back(level[j]);
      }
      p->rp[(size_t)i + 1] = (int32_t)p->ci.size();
    }

    if (bilu::complete_pattern(p, row_ptr, col_idx) != BILU_OK) {
      delete p;
      return BILU_ERR_OOM;
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return BILU_ERR_OOM;
  }
  *out = p;
  return BILU_OK;
}

// P'^T for the adjoint solve with A^T (its lower part is the transpose of U',
// its upper part the transpose of L), with Eq. 4 levels and the map from each
// of its factor slots to the slot of P' that holds the block to transpose.
extern "C" int bilu_pattern_transpose(const bilu_pattern* p, bilu_pattern** out) {
  if (!p || !out || p->is_transpose) return BILU_ERR_ARG;
  *out = nullptr;
  const int st = bilu::ensure_host(p);
  if (st != BILU_OK) return st;
  bilu_pattern* q = new (std::nothrow) bilu_pattern();
  if (!q) return BILU_ERR_OOM;
  try {
    const int32_t n = p->n;
    const size_t nnz = p->ci.size();
    q->n = n;
    q->k = p->k;
    q->nnz_a = p->nnz_a;
    q->is_transpose = true;
    // CSR transpose of P' (and of the entry levels); src[t'] = entry of P'
    q->rp.assign((size_t)n + 1, 0);
    for (size_t t = 0; t < nnz; ++t) ++q->rp[(size_t)p->ci[t] + 1];
    for (int32_t i = 0; i < n; ++i) q->rp[(size_t)i + 1] += q->rp[i];
    q->ci.resize(nnz);
    q->lev.resize(nnz);
    std::vector<int32_t> src(nnz), at(q->rp.begin(), q->rp.end() - 1);
    for (int32_t i = 0; i < n; ++i)
      for (int32_t t = p->rp[i]; t < p->rp[i + 1]; ++t) {
        const int32_t d = at[p->ci[t]]++;
        q->ci[d] = i;
        q->lev[d] = p->lev[t];
        src[d] = t;
      }
    finish_pattern(q);
    // factor slot of every P' entry: [L | D | U] positions
    auto slots = [](const bilu_pattern* m, std::vector<int32_t>& slot) {
      slot.resize(m->ci.size());
      const int64_t nl = m->nnz_l();
      for (int32_t i = 0; i < m->n; ++i) {
        int32_t a = m->lrp[i], c = m->urp[i];
        for (int32_t t = m->rp[i]; t < m->rp[i + 1]; ++t) {
          const int32_t j = m->ci[t];
          slot[t] = j < i ? a++ : (j == i ? (int32_t)(nl + i) : (int32_t)(nl + m->n + c++));
        }
      }
    };
    std::vector<int32_t> sp, sq;
    slots(p, sp);
    slots(q, sq);
    q->slot_src.assign((size_t)q->nslots(), -1);
    for (size_t d = 0; d < nnz; ++d) q->slot_src[(size_t)sq[d]] = sp[(size_t)src[d]];
  } catch (const std::bad_alloc&) {
    delete q;
    return BILU_ERR_OOM;
  }
  *out = q;
  return BILU_OK;
}

// Transpose of a block CSR pattern (host): row_ptr_t / col_idx_t of A^T and,
// for every block of A^T, the block of A it transposes.
extern "C" int bsr_transpose_pattern(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                     int32_t* row_ptr_t, int32_t* col_idx_t, int32_t* perm) {
  if (n < 0 || !row_ptr || !row_ptr_t || (n > 0 && row_ptr[n] > 0 && (!col_idx || !col_idx_t || !perm)))
    return BILU_ERR_ARG;
  if (row_ptr[0] != 0) return BILU_ERR_PATTERN;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return BILU_ERR_PATTERN;
  const int32_t nnz = n > 0 ? row_ptr[n] : 0;
  for (int32_t t = 0; t < nnz; ++t)
    if (col_idx[t] < 0 || col_idx[t] >= n) return BILU_ERR_PATTERN;
  std::fill(row_ptr_t, row_ptr_t + (size_t)n + 1, 0);
  for (int32_t t = 0; t < nnz; ++t) ++row_ptr_t[col_idx[t] + 1];
  for (int32_t i = 0; i < n; ++i) row_ptr_t[i + 1] += row_ptr_t[i];
  try {
    std::vector<int32_t> at(row_ptr_t, row_ptr_t + n);
    for (int32_t i = 0; i < n; ++i)
      for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
        const int32_t d = at[col_idx[t]]++;
        col_idx_t[d] = i;
        perm[d] = t;
      }
  } catch (const std::bad_alloc&) {
    return BILU_ERR_OOM;
  }
  return BILU_OK;
}

extern "C" int bilu_pattern_query(const bilu_pattern* p, bilu_pattern_info* info) {
  if (!p || !info) return BILU_ERR_ARG;
  info->n = p->n;
  info->k = p->k;
  info->nnz_a = p->nnz_a;
  info->nnz_p = p->cnt_p;
  info->nnz_l = p->nnz_l();
  info->nnz_u = p->nnz_u();
  info->nlev_l = p->nlev_l;
  info->nlev_u = p->nlev_u;
  return BILU_OK;
}

extern "C" int bilu_pattern_export(const bilu_pattern* p, int32_t* row_ptr, int32_t* col_idx,
                                   int32_t* lev, int32_t* lvl_lower, int32_t* lvl_upper) {
  if (!p) return BILU_ERR_ARG;
  const int st = bilu::ensure_host(p);
  if (st != BILU_OK) return st;
  const size_t n = (size_t)p->n, nnz = p->ci.size();
  if (row_ptr) std::memcpy(row_ptr, p->rp.data(), sizeof(int32_t) * (n + 1));
  if (col_idx && nnz) std::memcpy(col_idx, p->ci.data(), sizeof(int32_t) * nnz);
  if (lev && nnz) std::memcpy(lev, p->lev.data(), sizeof(int32_t) * nnz);
  if (lvl_lower && n) std::memcpy(lvl_lower, p->lvl_l.data(), sizeof(int32_t) * n);
  if (lvl_upper && n) std::memcpy(lvl_upper, p->lvl_u.data(), sizeof(int32_t) * n);
  return BILU_OK;
}

namespace bilu {

// Schedule of the sync-free triangular solves and factorization.
//
// Chunks.  Rows are cut into chunks of consecutive rows, about `target` rows
// each; the lower solve and the factorization walk chunks in ascending order,
// the upper solve in descending order.  The gap of a row r is the distance to
// its nearest dependency below it, r - max{j < r in L(r)} (and, for U',
// min{j > r-1 in U(r-1)} - (r-1); the smaller of the two counts).  A cut is
// placed before the row of largest gap > 1 in [target/2, 3*target/2] rows (at
// most 1024) from the chunk's start, the one nearest to `target` among equal
// gaps; else at `target`.  (Chunks stay within 1.5x the target: every CTA
// reserves shared memory for the longest one.)  In a natural grid ordering the rows of gap > 1
// start grid lines and the largest gaps start planes, so chunks hold whole
// lines and never straddle a plane: the chain along a line never crosses a
// chunk boundary (a chunk cut inside a line would wait for the previous
// chunk's last row before its first row could start), and no chunk mixes the
// end of one plane with the start of the next (whose rows become ready a
// whole plane apart, holding the chunk's CTA in between).
//
// Order inside a chunk.  The local level of a row is 1 + the largest local
// level of the rows of the same chunk it depends on (0 if none), i.e. Eq. 4
// restricted to the chunk; rows are listed by (local level, row) for L and
// (local level, descending row) for U'.  Chunk [lo, hi) occupies positions
// [lo, hi) of ord_l and of ord_u.
//
// Tickets hand chunks out in a topological order of the chunk dependency
// graph (a chunk depends on every other chunk holding a row one of its rows
// depends on), so a chunk only ever waits on chunks of smaller tickets.  The
// order is built by list scheduling: among the chunks whose predecessors are
// all listed, the next ticket goes to the one whose earliest row has the
// smallest Eq. 4 level (then the smaller chunk index).  The Eq. 4 level of a
// row is where it sits on the longest dependency chain, i.e. roughly when it
// can start, so chunks are claimed in about the order they can run and few
// resident CTAs sit on chunks that cannot start yet.  Chunk numbers: lower
// chunk c is bnd[c]..bnd[c+1]; upper chunk c is lower chunk nchunks-1-c.
void schedule_cuts(int32_t n, int32_t target, bool upper, const std::vector<int32_t>& gapl,
                   const std::vector<int32_t>& gapu, bilu_chunk_schedule* s) {
  auto gap = [&](int32_t r) -> int64_t {  // 0 < r < n; INT32_MAX: no dependency that side
    int64_t g = gapl[(size_t)r];
    if (upper) g = std::min<int64_t>(g, gapu[(size_t)r]);
    return g;
  };
  s->bnd.clear();
  s->bnd.push_back(0);
  int32_t max_len = 0;
  for (int32_t lo = 0; lo < n;) {
    int32_t hi = (int32_t)std::min<int64_t>(n, (int64_t)lo + target);
    if (hi < n) {
      const int32_t a = lo + std::max(1, target / 2);
      const int32_t z = (int32_t)std::min<int64_t>({(int64_t)n - 1, (int64_t)lo + target + target / 2,
                                                    (int64_t)lo + 1024});
      int32_t best = -1;
      int64_t best_gap = 1;
      for (int32_t r = a; r <= z; ++r) {
        const int64_t g = gap(r);
        if (g <= 1 || g < best_gap) continue;  // gap 1: r depends on r - 1
        if (g > best_gap || std::abs(r - (lo + target)) < std::abs(best - (lo + target))) {
          best = r;
          best_gap = g;
        }
      }
      if (best > lo) hi = best;
    }
    max_len = std::max(max_len, hi - lo);
    s->bnd.push_back(hi);
    lo = hi;
  }
  s->nchunks = (int32_t)s->bnd.size() - 1;
  s->max_len = max_len;
}

void ticket_order_lists(int32_t nchunks, const std::vector<int32_t>& prio, const std::vector<int64_t>& pred_ptr,
                        const std::vector<int32_t>& pred, std::vector<int32_t>& tick) {
  // successor lists (CSR by predecessor) and in-degrees from the predecessor lists
  std::vector<int64_t> off((size_t)nchunks + 1, 0);
  std::vector<int32_t> indeg((size_t)nchunks, 0);
  for (int32_t c = 0; c < nchunks; ++c) {
    indeg[c] = (int32_t)(pred_ptr[(size_t)c + 1] - pred_ptr[c]);
    for (int64_t e = pred_ptr[c]; e < pred_ptr[(size_t)c + 1]; ++e) ++off[(size_t)pred[e] + 1];
  }
  for (int32_t c = 0; c < nchunks; ++c) off[c + 1] += off[c];
  std::vector<int32_t> succ((size_t)off[nchunks]);
  {
    std::vector<int64_t> at(off.begin(), off.end() - 1);
    for (int32_t c = 0; c < nchunks; ++c)
      for (int64_t e = pred_ptr[c]; e < pred_ptr[(size_t)c + 1]; ++e) succ[at[pred[e]]++] = c;
  }
  std::priority_queue<std::pair<int32_t, int32_t>, std::vector<std::pair<int32_t, int32_t>>,
                      std::greater<std::pair<int32_t, int32_t>>>
      ready;
  for (int32_t c = 0; c < nchunks; ++c)
    if (indeg[c] == 0) ready.emplace(prio[c], c);
  tick.clear();
  tick.reserve((size_t)nchunks);
  while (!ready.empty()) {
    const int32_t c = ready.top().second;
    ready.pop();
    tick.push_back(c);
    for (int64_t e = off[c]; e < off[c + 1]; ++e)
      if (--indeg[succ[e]] == 0) ready.emplace(prio[succ[e]], succ[e]);
  }
  // a chunk depends only on chunks earlier in solve order: every chunk is listed
}

void build_schedule(const bilu_pattern* p, int32_t target, bool upper, bilu_chunk_schedule* s) {
  const int32_t n = p->n;
  // chunk boundaries from the gaps: r - (last column of L(r)), and the first
  // column of U'(r - 1) - (r - 1)
  std::vector<int32_t> gapl((size_t)n, INT32_MAX), gapu((size_t)n, INT32_MAX);
  for (int32_t r = 0; r < n; ++r) {
    if (p->lrp[r + 1] > p->lrp[r]) gapl[r] = r - p->lci[p->lrp[r + 1] - 1];
    if (r > 0 && p->urp[r] > p->urp[r - 1]) gapu[r] = p->uci[p->urp[r - 1]] - (r - 1);
  }
  schedule_cuts(n, target, upper, gapl, gapu, s);
  const int32_t nchunks = s->nchunks;
  const int32_t max_len = s->max_len;
  std::vector<int32_t> chunk_of((size_t)n);
  for (int32_t c = 0; c < nchunks; ++c)
    for (int32_t i = s->bnd[c]; i < s->bnd[c + 1]; ++i) chunk_of[i] = c;

  s->ord_l.assign((size_t)n, 0);
  s->ord_u.assign(upper ? (size_t)n : 0, 0);
  std::vector<int32_t> loc((size_t)std::max(max_len, 1), 0);
  std::vector<std::pair<int32_t, int32_t>> key;
  for (int32_t c = 0; c < nchunks; ++c) {
    const int32_t lo = s->bnd[c], hi = s->bnd[c + 1];
    key.clear();
    for (int32_t i = lo; i < hi; ++i) {
      int32_t l = 0;
      for (int32_t t = p->lrp[i]; t < p->lrp[i + 1]; ++t)
        if (p->lci[t] >= lo) l = std::max(l, loc[p->lci[t] - lo] + 1);
      loc[i - lo] = l;
      key.emplace_back(l, i);
    }
    std::sort(key.begin(), key.end());
    for (size_t q = 0; q < key.size(); ++q) s->ord_l[(size_t)lo + q] = key[q].second;
    if (!upper) continue;
    key.clear();
    for (int32_t i = hi - 1; i >= lo; --i) {
      int32_t l = 0;
      for (int32_t t = p->urp[i]; t < p->urp[i + 1]; ++t)
        if (p->uci[t] < hi) l = std::max(l, loc[p->uci[t] - lo] + 1);
      loc[i - lo] = l;
      key.emplace_back(l, -i);
    }
    std::sort(key.begin(), key.end());
    for (size_t q = 0; q < key.size(); ++q) s->ord_u[(size_t)lo + q] = -key[q].second;
  }
  // ticket orders (list scheduling over the chunk dependency graph)
  auto ticket_order = [&](bool up, std::vector<int32_t>& tick) {
    const std::vector<int32_t>& rpv = up ? p->urp : p->lrp;
    const std::vector<int32_t>& civ = up ? p->uci : p->lci;
    const std::vector<int32_t>& lvl = up ? p->lvl_u : p->lvl_l;
    std::vector<int32_t> prio((size_t)nchunks, 0), seen((size_t)nchunks, -1), pred;
    std::vector<int64_t> pred_ptr((size_t)nchunks + 1, 0);  // distinct predecessors (solve-order numbers)
    for (int32_t c = 0; c < nchunks; ++c) {
      const int32_t lc = up ? nchunks - 1 - c : c;  // the chunk's rows
      const int32_t lo = s->bnd[lc], hi = s->bnd[lc + 1];
      int32_t pm = INT32_MAX;
      for (int32_t i = lo; i < hi; ++i) {
        pm = std::min(pm, lvl.empty() ? 0 : lvl[i]);
        for (int32_t t = rpv[i]; t < rpv[i + 1]; ++t) {
          const int32_t j = civ[t];
          if (j >= lo && j < hi) continue;
          const int32_t cj = up ? nchunks - 1 - chunk_of[j] : chunk_of[j];
          if (seen[cj] == c) continue;
          seen[cj] = c;
          pred.push_back(cj);
        }
      }
      prio[c] = pm;
      pred_ptr[(size_t)c + 1] = (int64_t)pred.size();
    }
    ticket_order_lists(nchunks, prio, pred_ptr, pred, tick);
  };
  ticket_order(false, s->tick_l);
  if (upper) ticket_order(true, s->tick_u);
  else s->tick_u.clear();
  s->chunk = target;
  s->upper = upper;
}

}  // namespace bilu
