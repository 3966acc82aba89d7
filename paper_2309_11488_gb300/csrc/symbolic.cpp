// Host symbolic analysis: pattern validation, level or colour schedule, the
// row permutation, the warp-sliced layouts of A, L and U and the ILU0 update
// lists.  Runs once per sparsity pattern; the paper reuses its analysis for
// the whole simulation because the pattern never changes (Section 4.4).
#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>
#include <queue>
#include <utility>

#include "opm_internal.h"

namespace opm {
namespace {

// Edge list of the symmetrised pattern (i-j whenever block (i,j) or (j,i)
// exists, i != j), as CSR.
void symmetrise(int32_t n, const int32_t *rowptr, const int32_t *colidx, std::vector<int64_t> &gp,
                std::vector<int32_t> &ga) {
  gp.assign((size_t)n + 1, 0);
  for (int32_t i = 0; i < n; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j != i) {
        gp[i + 1]++;
        gp[j + 1]++;
      }
    }
  for (int32_t i = 0; i < n; ++i) gp[i + 1] += gp[i];
  ga.resize((size_t)gp[n]);
  std::vector<int64_t> fill(gp.begin(), gp.end() - 1);
  for (int32_t i = 0; i < n; ++i)
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j != i) {
        ga[fill[i]++] = j;
        ga[fill[j]++] = i;
      }
    }
}

// Level of a row: 0 without an earlier neighbour, else one more than the
// deepest earlier neighbour.  Rows of equal level share no edge.
int32_t level_sets(int32_t n, const std::vector<int64_t> &gp, const std::vector<int32_t> &ga,
                   std::vector<int32_t> &key) {
  key.assign(n, 0);
  int32_t nsets = n > 0 ? 1 : 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int64_t m = gp[i]; m < gp[i + 1]; ++m) {
      int32_t j = ga[m];
      if (j < i) l = std::max(l, key[j] + 1);
    }
    key[i] = l;
    nsets = std::max(nsets, l + 1);
  }
  return nsets;
}

// Greedy first-fit colouring in natural order: each row takes the smallest
// colour that no earlier neighbour holds.
int32_t colour_sets(int32_t n, const std::vector<int64_t> &gp, const std::vector<int32_t> &ga,
                    std::vector<int32_t> &key) {
  key.assign(n, -1);
  std::vector<int32_t> stamp;
  int32_t nsets = n > 0 ? 1 : 0;
  for (int32_t i = 0; i < n; ++i) {
    for (int64_t m = gp[i]; m < gp[i + 1]; ++m) {
      int32_t c = key[ga[m]];
      if (c >= 0) {
        if ((size_t)c >= stamp.size()) stamp.resize((size_t)c + 1, -1);
        stamp[c] = i;
      }
    }
    int32_t c = 0;
    while ((size_t)c < stamp.size() && stamp[c] == i) ++c;
    key[i] = c;
    nsets = std::max(nsets, c + 1);
  }
  return nsets;
}

// Greedy first-fit colouring in smallest-last order (Matula & Beck): rows
// are removed one at a time, each time one of least degree among those left
// (distinct neighbours still present; ties to the lowest row), then coloured
// in the reverse order of removal.
// Each row's distinct neighbours, sorted.
void distinct_lists(int32_t n, const std::vector<int64_t> &gp, const std::vector<int32_t> &ga,
                    std::vector<int64_t> &dp, std::vector<int32_t> &da) {
  dp.assign((size_t)n + 1, 0);
  da.clear();
  da.reserve(ga.size());
  std::vector<int32_t> tmp;
  for (int32_t i = 0; i < n; ++i) {
    tmp.assign(ga.begin() + gp[i], ga.begin() + gp[i + 1]);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    da.insert(da.end(), tmp.begin(), tmp.end());
    dp[i + 1] = (int64_t)da.size();
  }
}

int32_t colour_sets_sl_lists(int32_t n, const std::vector<int64_t> &dp, const std::vector<int32_t> &da,
                             std::vector<int32_t> &key);

int32_t colour_sets_sl(int32_t n, const std::vector<int64_t> &gp, const std::vector<int32_t> &ga,
                       std::vector<int32_t> &key) {
  std::vector<int64_t> dp;
  std::vector<int32_t> da;
  distinct_lists(n, gp, ga, dp, da);
  return colour_sets_sl_lists(n, dp, da, key);
}

int32_t colour_sets_sl_lists(int32_t n, const std::vector<int64_t> &dp, const std::vector<int32_t> &da,
                             std::vector<int32_t> &key) {
  std::vector<int32_t> deg(n), order;
  order.reserve(n);
  std::vector<char> gone(n, 0);
  std::priority_queue<int64_t, std::vector<int64_t>, std::greater<int64_t>> heap;
  for (int32_t i = 0; i < n; ++i) {
    deg[i] = (int32_t)(dp[i + 1] - dp[i]);
    heap.push(((int64_t)deg[i] << 32) | i);
  }
  while (!heap.empty()) {
    const int64_t k = heap.top();
    heap.pop();
    const int32_t v = (int32_t)(k & 0xffffffff), d = (int32_t)(k >> 32);
    if (gone[v] || d != deg[v]) continue;  // stale entry
    gone[v] = 1;
    order.push_back(v);
    for (int64_t m = dp[v]; m < dp[v + 1]; ++m) {
      const int32_t u = da[m];
      if (!gone[u]) heap.push(((int64_t)(--deg[u]) << 32) | u);
    }
  }
  key.assign(n, -1);
  std::vector<int32_t> stamp((size_t)n + 1, -1);
  int32_t nsets = n > 0 ? 1 : 0;
  for (auto it = order.rbegin(); it != order.rend(); ++it) {
    const int32_t v = *it;
    for (int64_t m = dp[v]; m < dp[v + 1]; ++m)
      if (key[da[m]] >= 0) stamp[key[da[m]]] = v;
    int32_t c = 0;
    while (stamp[c] == v) ++c;
    key[v] = c;
    nsets = std::max(nsets, c + 1);
  }
  return nsets;
}

// Smallest-last colouring, then fewer colour classes by Kempe-chain
// exchanges (Kempe 1879): while more than two colours remain, each row v of
// the highest colour t (in row order) takes the smallest lower colour free
// among its neighbours, or else, trying colour pairs (a, b) below t with a
// then b ascending, the first pair whose Kempe chain is usable: the rows
// reached breadth first from v's a-coloured neighbours (in list order)
// through rows coloured a or b.  The chain is usable when the search meets
// no other neighbour of v within kKempeCap rows; a and b are then swapped
// on it (the colouring stays proper and no neighbour of v keeps a) and v
// takes a.  The pass stops at the first class that cannot be emptied.
constexpr int32_t kKempeCap = 16384;

int32_t colour_sets_kempe(int32_t n, const std::vector<int64_t> &gp, const std::vector<int32_t> &ga,
                          std::vector<int32_t> &key) {
  std::vector<int64_t> dp;
  std::vector<int32_t> da;
  distinct_lists(n, gp, ga, dp, da);
  int32_t ncol = colour_sets_sl_lists(n, dp, da, key);
  std::vector<int32_t> owner(n, -1), seen(n, -1), chain;
  chain.reserve(kKempeCap);
  std::vector<char> taken;
  int32_t search = 0;
  // the Kempe chain of (a, b) from v's a-neighbours; false when unusable
  auto collect = [&](int32_t v, int32_t a, int32_t b) {
    ++search;
    chain.clear();
    for (int64_t m = dp[v]; m < dp[v + 1]; ++m) {
      const int32_t u = da[m];
      if (key[u] != a) continue;
      if ((int32_t)chain.size() == kKempeCap) return false;
      seen[u] = search;
      chain.push_back(u);
    }
    for (size_t h = 0; h < chain.size(); ++h) {
      const int32_t x = chain[h];
      for (int64_t m = dp[x]; m < dp[x + 1]; ++m) {
        const int32_t y = da[m];
        if (seen[y] == search || (key[y] != a && key[y] != b)) continue;
        if (owner[y] == v || (int32_t)chain.size() == kKempeCap) return false;
        seen[y] = search;
        chain.push_back(y);
      }
    }
    return true;
  };
  while (ncol > 2) {
    const int32_t t = ncol - 1;
    bool emptied = true;
    for (int32_t v = 0; v < n; ++v) {
      if (key[v] != t) continue;
      taken.assign((size_t)t, 0);
      for (int64_t m = dp[v]; m < dp[v + 1]; ++m) {
        owner[da[m]] = v;
        if (key[da[m]] < t) taken[key[da[m]]] = 1;
      }
      const int32_t lowest = (int32_t)(std::find(taken.begin(), taken.end(), 0) - taken.begin());
      if (lowest < t) {
        key[v] = lowest;
        continue;
      }
      bool moved = false;
      for (int32_t a = 0; a < t && !moved; ++a)
        for (int32_t b = 0; b < t && !moved; ++b) {
          if (b == a || !collect(v, a, b)) continue;
          for (int32_t x : chain) key[x] = key[x] == a ? b : a;
          key[v] = a;
          moved = true;
        }
      if (!moved) emptied = false;
    }
    if (!emptied) break;
    --ncol;
  }
  return ncol;
}

// Warp-sliced order of a CSR part: fills pos[csr block] = sliced block index
// and slot[csr block] = packed value location.
void slice_layout(int32_t n, const std::vector<int32_t> &rp, std::vector<int64_t> &pos,
                  std::vector<int64_t> &slot, int64_t val_base) {
  int64_t nnz = rp[n];
  pos.assign((size_t)nnz, 0);
  slot.assign((size_t)nnz, 0);
  for (int32_t r0 = 0; r0 < n; r0 += kWarp) {
    int32_t r1 = std::min(n, r0 + kWarp);
    int32_t maxlen = 0;
    for (int32_t i = r0; i < r1; ++i) maxlen = std::max(maxlen, rp[i + 1] - rp[i]);
    int64_t base = rp[r0];
    for (int32_t k = 0; k < maxlen; ++k) {
      int32_t cnt = 0;
      for (int32_t i = r0; i < r1; ++i)
        if (rp[i + 1] - rp[i] > k) ++cnt;
      int32_t q = 0;
      for (int32_t i = r0; i < r1; ++i)
        if (rp[i + 1] - rp[i] > k) {
          int64_t c = rp[i] + k;
          pos[c] = base + q;
          slot[c] = slot_pack(val_base + 9 * base + q, cnt);
          ++q;
        }
      base += cnt;
    }
  }
}

}  // namespace

opm_status analyse(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *part,
                   int32_t schedule, Analysis &an, int32_t *err_row) {
  *err_row = -1;
  if (n < 0) return OPM_ERR_ARG;
  if (rowptr[0] != 0) {
    *err_row = 0;
    return OPM_ERR_PATTERN;
  }
  for (int32_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) {
      *err_row = i;
      return OPM_ERR_PATTERN;
    }
  }
  const int64_t nnzb = rowptr[n];
  if (9 * (nnzb + (int64_t)n + kWarp) >= ((int64_t)1 << 31)) return OPM_ERR_ARG;  // int32 value offsets
  for (int32_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
      int32_t j = colidx[m];
      if (j < 0 || j >= n || (m > rowptr[i] && colidx[m - 1] >= j)) {
        *err_row = i;
        return OPM_ERR_PATTERN;
      }
      diag |= (j == i);
    }
    if (!diag) {
      *err_row = i;
      return OPM_ERR_NO_DIAG;
    }
  }

  an = Analysis();
  an.n = n;
  an.nnzb = nnzb;
  if (schedule == OPM_SCHED_AUTO) schedule = OPM_SCHED_COLOUR_KEMPE;
  an.schedule = schedule;

  // ---- the preconditioner's pattern.  With a partition (block-Jacobi ILU0,
  // Section 4.5) only the blocks joining two rows of the same partition are
  // factorised; the SpMV keeps every block.  Schedule, factors, phases and
  // update lists all follow this pattern (mrp, mci; the full one otherwise).
  std::vector<char> keep((size_t)nnzb, 1);
  std::vector<int32_t> jrp, jci;
  const int32_t *mrp = rowptr, *mci = colidx;
  if (part) {
    jrp.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
      for (int64_t m = rowptr[i]; m < rowptr[i + 1]; ++m) {
        keep[m] = part[i] == part[colidx[m]];
        if (keep[m]) jci.push_back(colidx[m]);
      }
      jrp[i + 1] = (int32_t)jci.size();
    }
    mrp = jrp.data();
    mci = jci.data();
    an.nnzb_kept = (int64_t)jci.size();
  } else {
    an.nnzb_kept = nnzb;
  }

  // ---- schedule and permutation (perm[new] = old, natural order inside a group)
  std::vector<int32_t> key;
  int32_t nkeys = 0;
  if (schedule == OPM_SCHED_NATURAL) {
    key.assign(n, 0);
    an.nsets = n > 0 ? 1 : 0;
    nkeys = an.nsets;
  } else {
    std::vector<int64_t> gp;
    std::vector<int32_t> ga;
    symmetrise(n, mrp, mci, gp, ga);
    an.nsets = schedule == OPM_SCHED_LEVEL       ? level_sets(n, gp, ga, key)
               : schedule == OPM_SCHED_COLOUR    ? colour_sets(n, gp, ga, key)
               : schedule == OPM_SCHED_COLOUR_SL ? colour_sets_sl(n, gp, ga, key)
                                                 : colour_sets_kempe(n, gp, ga, key);
    // Inside a set, rows with no neighbour in a later set (hence no U block)
    // come first: they finish within the forward sweep, and the backward
    // sweep of the set covers a contiguous tail.  Rows of a set share no
    // edge, so their order does not change the factors.
    // Inside each of those two groups the few rows longer than the most
    // common row length (fault connections, ties to the smaller length) go
    // last, so that most warps hold rows of nearly equal length.
    std::vector<int64_t> hist;
    for (int32_t i = 0; i < n; ++i) {
      const int32_t len = mrp[i + 1] - mrp[i];
      if ((size_t)len >= hist.size()) hist.resize((size_t)len + 1, 0);
      hist[len]++;
    }
    const int32_t common = (int32_t)(std::max_element(hist.begin(), hist.end()) - hist.begin());
    std::vector<int32_t> sub(n);
    for (int32_t i = 0; i < n; ++i) {
      bool open = false;
      for (int64_t m = gp[i]; m < gp[i + 1] && !open; ++m) open = key[ga[m]] > key[i];
      const bool longer = mrp[i + 1] - mrp[i] > common;
      sub[i] = 2 * (2 * key[i] + (open ? 1 : 0)) + (longer ? 1 : 0);
    }
    key.swap(sub);
    nkeys = 4 * an.nsets;
  }
  std::vector<int64_t> count((size_t)nkeys + 1, 0);
  for (int32_t i = 0; i < n; ++i) count[key[i] + 1]++;
  for (int32_t s = 0; s < nkeys; ++s) count[s + 1] += count[s];
  an.perm.resize(n);
  an.iperm.resize(n);
  for (int32_t i = 0; i < n; ++i) {
    int32_t ni = (int32_t)count[key[i]]++;
    an.perm[ni] = i;
    an.iperm[i] = ni;
  }

  // ---- permuted CSR with sorted columns and the caller's block index
  std::vector<int32_t> &arp = an.a_rowptr;
  arp.assign((size_t)n + 1, 0);
  for (int32_t ni = 0; ni < n; ++ni) arp[ni + 1] = arp[ni] + (rowptr[an.perm[ni] + 1] - rowptr[an.perm[ni]]);
  std::vector<int32_t> pcol((size_t)nnzb), psrc((size_t)nnzb);
  std::vector<char> pk((size_t)nnzb);  // block kept in the preconditioner
  std::vector<std::pair<int32_t, int32_t>> tmp;
  an.l_rowptr.assign((size_t)n + 1, 0);
  an.u_rowptr.assign((size_t)n + 1, 0);
  for (int32_t ni = 0; ni < n; ++ni) {
    int32_t oi = an.perm[ni];
    tmp.clear();
    for (int64_t m = rowptr[oi]; m < rowptr[oi + 1]; ++m) tmp.emplace_back(an.iperm[colidx[m]], (int32_t)m);
    std::sort(tmp.begin(), tmp.end());
    int32_t nl = 0, nu = 0;
    for (size_t q = 0; q < tmp.size(); ++q) {
      pcol[arp[ni] + q] = tmp[q].first;
      psrc[arp[ni] + q] = tmp[q].second;
      pk[arp[ni] + q] = keep[tmp[q].second];
      if (!keep[tmp[q].second]) continue;
      nl += tmp[q].first < ni;
      nu += tmp[q].first > ni;
    }
    an.l_rowptr[ni + 1] = an.l_rowptr[ni] + nl;
    an.u_rowptr[ni + 1] = an.u_rowptr[ni] + nu;
    an.max_row_len = std::max<int32_t>(an.max_row_len, (int32_t)tmp.size());
  }
  an.nnz_l = an.l_rowptr[n];
  an.nnz_u = an.u_rowptr[n];
  {
    const int64_t ns = ((int64_t)n + kWarp - 1) / kWarp;
    an.sl_mask.assign((size_t)(2 * ns), 0u);
    std::vector<char> read_later((size_t)n, 0);
    for (int32_t ni = 0; ni < n; ++ni)
      for (int64_t c = arp[ni]; c < arp[ni + 1] && pcol[c] < ni; ++c)
        if (pk[c]) read_later[pcol[c]] = 1;
    for (int32_t ni = 0; ni < n; ++ni) {
      const bool no_u = an.u_rowptr[ni + 1] == an.u_rowptr[ni];
      const uint32_t bit = 1u << (ni % kWarp);
      if (no_u) an.sl_mask[2 * (ni / kWarp)] |= bit;
      if (!no_u || read_later[ni]) an.sl_mask[2 * (ni / kWarp) + 1] |= bit;
    }
  }

  // ---- warp-sliced layouts.  Factor values: [L | U | Dinv slices].
  std::vector<int64_t> a_pos, a_slot, l_pos, l_slot, u_pos, u_slot;
  slice_layout(n, arp, a_pos, a_slot, 0);
  slice_layout(n, an.l_rowptr, l_pos, l_slot, 0);
  slice_layout(n, an.u_rowptr, u_pos, u_slot, 9 * an.nnz_l);
  an.d_off = 9 * (an.nnz_l + an.nnz_u);
  const int64_t nslices = ((int64_t)n + kWarp - 1) / kWarp;
  an.lu_vals = an.d_off + kSliceVals * nslices;
  auto d_slot = [&](int32_t i) { return slot_pack(an.d_off + kSliceVals * (i / kWarp) + (i % kWarp), kWarp); };

  an.a_col.assign((size_t)nnzb, 0);
  an.a_src.assign((size_t)nnzb, 0);
  an.a_dst.assign((size_t)nnzb, 0);
  an.a_csr_slot.assign((size_t)nnzb, 0);
  an.l_col.assign((size_t)an.nnz_l, 0);
  an.u_col.assign((size_t)an.nnz_u, 0);
  std::vector<int64_t> a_at((size_t)nnzb);  // sliced A position of permuted CSR block c
  for (int32_t ni = 0; ni < n; ++ni) {
    int64_t lc = an.l_rowptr[ni], uc = an.u_rowptr[ni];
    int64_t cd = arp[ni];
    while (pcol[cd] != ni) ++cd;  // every row holds its diagonal (checked above)
    for (int64_t c = arp[ni]; c < arp[ni + 1]; ++c) {
      // A's order inside the row: the diagonal first, then column order
      const int64_t rank = c == cd ? 0 : (c - arp[ni]) + (c < cd ? 1 : 0);
      a_at[c] = a_pos[arp[ni] + rank];
      int32_t j = pcol[c];
      int64_t dst;
      if (!pk[c]) {
        dst = -1;  // outside the preconditioner: no factor slot
      } else if (j < ni) {
        an.l_col[l_pos[lc]] = j;
        dst = l_slot[lc++];
      } else if (j > ni) {
        an.u_col[u_pos[uc]] = j;
        dst = u_slot[uc++];
      } else {
        dst = d_slot(ni);
      }
      an.a_col[a_at[c]] = j;
      an.a_src[a_at[c]] = psrc[c];
      an.a_dst[a_at[c]] = dst;
      an.a_csr_slot[c] = dst;
    }
  }

  // ---- phases.  Row i opens a new phase when it reads a row of the current
  // run in the forward sweep (an L column >= start) or when an earlier row of
  // the run reads it in the backward sweep (a U column of the run == i).
  an.phase_ptr.assign(1, 0);
  {
    int32_t start = 0, limit = INT32_MAX;
    for (int32_t i = 0; i < n; ++i) {
      bool split = i >= limit;
      for (int64_t c = arp[i]; c < arp[i + 1] && !split; ++c)
        if (pk[c] && pcol[c] < i && pcol[c] >= start) split = true;
      if (split && i > start) {
        an.phase_ptr.push_back(i);
        start = i;
        limit = INT32_MAX;
      }
      for (int64_t c = arp[i]; c < arp[i + 1]; ++c)
        if (pk[c] && pcol[c] > i) limit = std::min(limit, pcol[c]);
    }
    if (n > 0) an.phase_ptr.push_back(n);
  }

  // ---- ILU0 update lists: for L block (i,k), every j > k present in row i
  // and in row k gives A_ij -= L_ik * U_kj (Algorithm 2's inner loop).  A row
  // all of whose products land on its diagonal block is walked in one pass
  // by the factorisation (fz_mask, a_aux).
  an.upd_ptr.assign((size_t)an.nnz_l + 1, 0);
  an.upd_dst.clear();
  an.upd_src.clear();
  an.a_aux.assign((size_t)nnzb, -1);
  an.fz_mask.assign((size_t)((n + kWarp - 1) / kWarp), 0u);
  std::vector<char> upper_hit((size_t)n, 0);  // some product lands on an upper block of the row
  for (int32_t ni = 0; ni < n; ++ni) {
    bool fused = true;
    int64_t lc = an.l_rowptr[ni];
    for (int64_t c = arp[ni]; c < arp[ni + 1] && pcol[c] < ni; ++c) {
      if (!pk[c]) continue;
      int32_t k = pcol[c];
      // row k's kept upper blocks (permuted CSR positions; ku counts them)
      int64_t ku = an.u_rowptr[k];
      int64_t kc = arp[k];
      while (kc < arp[k + 1] && pcol[kc] <= k) ++kc;  // first upper block of row k
      while (kc < arp[k + 1] && !pk[kc]) ++kc;
      int64_t ic = c + 1;
      while (ic < arp[ni + 1] && !pk[ic]) ++ic;
      while (ic < arp[ni + 1] && kc < arp[k + 1]) {
        if (pcol[ic] < pcol[kc]) {
          do ++ic; while (ic < arp[ni + 1] && !pk[ic]);
        } else if (pcol[ic] > pcol[kc]) {
          do ++kc; while (kc < arp[k + 1] && !pk[kc]);
          ++ku;
        } else {
          an.upd_dst.push_back(an.a_csr_slot[ic]);
          an.upd_src.push_back(u_slot[ku]);
          if (pcol[ic] == ni) an.a_aux[a_at[c]] = u_slot[ku];
          else fused = false;
          if (pcol[ic] > ni) upper_hit[ni] = 1;
          do ++ic; while (ic < arp[ni + 1] && !pk[ic]);
          do ++kc; while (kc < arp[k + 1] && !pk[kc]);
          ++ku;
        }
      }
      an.upd_ptr[lc + 1] = (int32_t)an.upd_dst.size();
      ++lc;
    }
    if (fused) {
      an.fz_mask[ni / kWarp] |= 1u << (ni % kWarp);
    } else {
      for (int64_t c = arp[ni]; c < arp[ni + 1]; ++c) an.a_aux[a_at[c]] = -1;
    }
  }
  if (an.upd_dst.size() >= ((size_t)1 << 31)) return OPM_ERR_ARG;
  an.nupd = (int64_t)an.upd_dst.size();

  // ---- what the products after an application walk (sp_mask, sp_len)
  an.sp_mask.assign((size_t)(2 * nslices), 0u);
  an.sp_len.assign((size_t)n, 0);
  an.nnzb_product = 0;
  an.rows_identity = 0;
  an.rows_reuse = 0;
  for (int32_t ni = 0; ni < n; ++ni) {
    int32_t lower = 0;
    bool all_kept = true, upper_kept = true, has_upper = false;
    for (int64_t c = arp[ni]; c < arp[ni + 1]; ++c) {
      lower += pcol[c] < ni;
      has_upper = has_upper || pcol[c] > ni;
      if (!pk[c]) {
        all_kept = false;
        if (pcol[c] > ni) upper_kept = false;
      }
    }
    const uint32_t bit = 1u << (ni % kWarp);
    int32_t len = arp[ni + 1] - arp[ni];
    if (lower == 0 && all_kept) {
      an.sp_mask[2 * (ni / kWarp)] |= bit;
      len = 0;
      ++an.rows_identity;
    } else if (has_upper && upper_kept && !upper_hit[ni]) {
      an.sp_mask[2 * (ni / kWarp) + 1] |= bit;
      len = 1 + lower;
      ++an.rows_reuse;
    }
    an.sp_len[ni] = len;
    an.nnzb_product += len;
  }
  an.sp_tile.assign((size_t)(((int64_t)n + kSpmvRows - 1) / kSpmvRows), 0);
  for (int32_t ni = 0; ni < n; ++ni) an.sp_tile[ni / kSpmvRows] += an.sp_len[ni];
  return OPM_OK;
}

}  // namespace opm
