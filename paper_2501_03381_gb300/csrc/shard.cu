// Host-only helpers for splitting one request over several processes (one
// GPU each) and merging what they return.  Nplets are independent (Methods,
// "Parallel and batched computation of HOI": the subsets are computed
// without interference), so a request shards into contiguous id ranges with
// no exchange until the per-order records are merged once at the end.
//
// Work model per nplet of order k: F(k) = 2/3 k^3 + 2 k^2 FLOP (one LDL^T,
// one unit-lower inverse, the inverse diagonal).  The partition works in
// units of F/3 so that the arithmetic is exact in 128-bit integers and gives
// the same bounds on every host.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "thoi.h"

namespace {

typedef unsigned __int128 u128;

uint64_t binom_u64(int n, int k) {
  if (k < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  u128 r = 1;
  for (int i = 1; i <= k; i++) r = r * (u128)(n - k + i) / (u128)i;
  return (uint64_t)r;
}

u128 work3(int k) { return (u128)(2ull * k * k * k + 6ull * k * k); }

struct Ent {
  double v;
  uint64_t id;
};

// Ordering of a top list: side 0 by (value desc, id asc), side 1 by
// (value asc, id asc).
bool ent_before(int side, const Ent& a, const Ent& b) {
  if (a.v != b.v) return side == 0 ? a.v > b.v : a.v < b.v;
  return a.id < b.id;
}

}  // namespace

extern "C" thoi_status thoi_partition(int64_t N, const int32_t* orders, int32_t n_orders,
                                      int32_t R, uint64_t* bounds) {
  if (N < 1 || N > THOI_MAX_N || !orders || n_orders < 1 || R < 1 || !bounds)
    return THOI_ERR_INVALID_ARG;
  std::vector<uint64_t> cnt(n_orders);
  u128 W = 0;
  for (int o = 0; o < n_orders; o++) {
    if (orders[o] < 1 || orders[o] > N) return THOI_ERR_INVALID_ARG;
    cnt[o] = binom_u64((int)N, orders[o]);
    W += (u128)cnt[o] * work3(orders[o]);
  }
  bounds[0] = 0;
  for (int r = 1; r <= R; r++) {
    // first id whose cumulative work reaches W * r / R
    const u128 target = W * (u128)r / (u128)R;
    u128 before = 0;
    uint64_t off = 0, id = 0;
    bool placed = false;
    for (int o = 0; o < n_orders && !placed; o++) {
      const u128 w = work3(orders[o]);
      const u128 span = (u128)cnt[o] * w;
      if (before + span >= target) {
        const u128 need = target - before;
        uint64_t q = (uint64_t)((need + w - 1) / w);
        if (q > cnt[o]) q = cnt[o];
        id = off + q;
        placed = true;
      }
      before += span;
      off += cnt[o];
    }
    if (!placed) id = off;
    bounds[r] = id < bounds[r - 1] ? bounds[r - 1] : id;
  }
  return THOI_OK;
}

extern "C" thoi_status thoi_merge_records(const void* in, int32_t R, int32_t n_orders,
                                          int32_t top_m, void* out) {
  if (!in || !out || R < 1 || n_orders < 1 || top_m < 0 || top_m > THOI_MAX_TOP_M)
    return THOI_ERR_INVALID_ARG;
  const size_t per = thoi_records_bytes(n_orders, top_m);
  const unsigned char* base = (const unsigned char*)in;
  unsigned char* ob = (unsigned char*)out;
  std::vector<thoi_order_record> recs((size_t)n_orders);
  std::vector<thoi_top_entry> tops((size_t)n_orders * 2 * top_m);
  for (int q = 0; q < n_orders; q++) {
    thoi_order_record M;
    memset(&M, 0, sizeof M);
    double wsum[5] = {0, 0, 0, 0, 0};
    uint64_t valid = 0;
    bool have = false;
    std::vector<Ent> cand[2];
    for (int r = 0; r < R; r++) {
      const unsigned char* blk = base + per * (size_t)r;
      thoi_order_record a;
      memcpy(&a, blk + (size_t)q * sizeof(thoi_order_record), sizeof a);
      if (r == 0) M.k = a.k;
      else if (a.k != M.k) return THOI_ERR_INVALID_ARG;
      M.count += a.count;
      M.count_neg_O += a.count_neg_O;
      M.n_refactored += a.n_refactored;
      M.n_not_pd += a.n_not_pd;
      const uint64_t c = a.count - a.n_not_pd;
      if (c == 0) continue;
      for (int m = 0; m < 5; m++) {
        wsum[m] += a.mean[m] * (double)c;
        if (!have || a.min[m] < M.min[m] || (a.min[m] == M.min[m] && a.argmin[m] < M.argmin[m])) {
          M.min[m] = a.min[m];
          M.argmin[m] = a.argmin[m];
        }
        if (!have || a.max[m] > M.max[m] || (a.max[m] == M.max[m] && a.argmax[m] < M.argmax[m])) {
          M.max[m] = a.max[m];
          M.argmax[m] = a.argmax[m];
        }
      }
      have = true;
      valid += c;
      const int n = a.top_count < top_m ? a.top_count : top_m;
      const unsigned char* tb = blk + (size_t)n_orders * sizeof(thoi_order_record) +
                                (size_t)q * 2 * top_m * sizeof(thoi_top_entry);
      for (int side = 0; side < 2; side++)
        for (int i = 0; i < n; i++) {
          thoi_top_entry e;
          memcpy(&e, tb + ((size_t)side * top_m + i) * sizeof e, sizeof e);
          cand[side].push_back(Ent{e.value, e.id});
        }
    }
    if (have) {
      for (int m = 0; m < 5; m++) M.mean[m] = wsum[m] / (double)valid;
    } else {
      for (int m = 0; m < 5; m++) M.argmin[m] = M.argmax[m] = ~0ull;
    }
    M.top_count = (int32_t)(valid < (uint64_t)top_m ? valid : (uint64_t)top_m);
    for (int side = 0; side < 2; side++) {
      std::vector<Ent>& v = cand[side];
      std::sort(v.begin(), v.end(), [side](const Ent& a, const Ent& b) { return ent_before(side, a, b); });
      for (int i = 0; i < top_m; i++) {
        thoi_top_entry& e = tops[((size_t)q * 2 + side) * top_m + i];
        if (i < M.top_count && i < (int)v.size()) {
          e.value = v[i].v;
          e.id = v[i].id;
        } else {
          e.value = 0.0;
          e.id = ~0ull;
        }
      }
    }
    recs[q] = M;
  }
  memcpy(ob, recs.data(), (size_t)n_orders * sizeof(thoi_order_record));
  if (top_m > 0)
    memcpy(ob + (size_t)n_orders * sizeof(thoi_order_record), tops.data(),
           tops.size() * sizeof(thoi_top_entry));
  return THOI_OK;
}
