// Launch plans: the default rule for a shape (tiles, group length, split count), the
// checks a plan must pass, and the buffer layout quantities that depend on the plan.  A
// plan depends on the shape only, never on the data or the load.
#include <algorithm>
#include <string>

#include "rsim_internal.h"

namespace rsim {

int tile_nt(int L) { return L >= 128 ? 128 : ((L + 7) / 8) * 8; }

int64_t tensor_split_stride(int V, int Ns, int L, int nt) {
  const int64_t mtiles = ((int64_t)V * Ns + 127) / 128;
  return mtiles * ((L + nt - 1) / nt) * 128 * nt;
}

bool uses_partial(int tier, int64_t P, int splits, int group) {
  if (tier == RSIM_TIER_NUFFT) return false;
  if (splits > 1) return true;
  if (tier == RSIM_TIER_FP32) return false;
  const int64_t chunks = (P + kChunkPx - 1) / kChunkPx;
  return chunks > group;
}

int group_chunks(int tier) {
  return (tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16) ? 40 : 96;
}

// The split tiers' 2e-5 bar leaves room for the round-toward-zero bias of at most 40
// chunks (480 accumulating MMAs, a relative shrink of about 1e-5); the plain 16-bit tiers
// (1e-2) allow 384 chunks (1536 MMAs, about 3e-5).
int group_chunks_max(int tier) {
  return (tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16) ? 40 : 384;
}

int units_per_split(int tier, int V, int Ns, int L, int tile_n) {
  if (tier == RSIM_TIER_FP32) return V * ((Ns + tile_n - 1) / tile_n) * ((L + kDirectTileL - 1) / kDirectTileL);
  const int64_t rows = (int64_t)V * Ns;
  const int nt = (L + tile_n - 1) / tile_n;
  return (int)(((rows + 127) / 128) * nt);
}

int default_splits(int tier, int V, int Ns, int L, int tile_n, int64_t P, int num_sms) {
  if (tier == RSIM_TIER_NUFFT) return 1;
  const int tiles = units_per_split(tier, V, Ns, L, tile_n);
  const int64_t chunks = (P + kChunkPx - 1) / kChunkPx;
  // keep at least 8 chunks (256 pixels) per split
  int64_t smax = chunks / 8 > 0 ? chunks / 8 : 1;
  if (smax > kMaxSplits) smax = kMaxSplits;
  if (tier == RSIM_TIER_FP32) {
    // FP32 accumulation: at most 8192 pixels per split, so that the running sum of
    // random-phase terms keeps a relative rounding error of a few 1e-6 (the splits are
    // then added with compensated sums); above that, the split count that fills whole
    // waves of two resident CTAs per SM best
    const int64_t smin = std::min<int64_t>(std::max<int64_t>((P + 8191) / 8192, 1), kMaxSplits);
    const int64_t slots = 2ll * num_sms;
    double best = -1.0;
    int64_t bs = smin;
    for (int64_t s = smin; s <= std::max(smin, smax); ++s) {
      const int64_t units = (int64_t)tiles * s;
      const int64_t waves = (units + slots - 1) / slots;
      const double eff = (double)units / (double)(waves * slots) - 0.001 * s;
      if (eff > best + 1e-9) {
        best = eff;
        bs = s;
      }
    }
    return (int)bs;
  }
  // tensor tiers: one persistent CTA per SM takes equal units from a counter; pick the
  // split count whose unit count fills whole rounds of SMs best, with a small cost per
  // split for the partial buffer it adds
  double best = -1.0;
  int bs = 1;
  for (int s = 1; s <= smax; ++s) {
    const int64_t units = (int64_t)tiles * s;
    const int64_t rounds = (units + num_sms - 1) / num_sms;
    const double eff = (double)units / (double)(rounds * num_sms) - 0.003 * s;
    if (eff > best + 1e-9) {
      best = eff;
      bs = s;
    }
  }
  return bs;
}

void resolve_tile(int tier, const Consts& k, rsim_plan* p) {
  if (tier == RSIM_TIER_FP32) {
    if (p->tile_n == 0) p->tile_n = kDirectTileN;
    p->group_chunks = 0;
  } else if (tensor_tier(tier)) {
    if (p->tile_n == 0) p->tile_n = tile_nt(k.L);
    if (p->group_chunks == 0) p->group_chunks = group_chunks(tier);
  } else {
    p->tile_n = 0;
    p->group_chunks = 0;
  }
  p->chunk_px = kChunkPx;
}

rsim_plan default_plan(int tier, const Consts& k, int64_t P, int num_sms) {
  rsim_plan p{};
  resolve_tile(tier, k, &p);
  p.splits = default_splits(tier, k.V, k.Ns, k.L, p.tile_n, P, num_sms);
  return p;
}

std::string plan_problem(int tier, const Consts& k, const rsim_plan& p) {
  if (p.splits < 1 || p.splits > kMaxSplits) return "plan splits must be in 1..64";
  if (p.grid < 0) return "plan grid must be >= 0";
  if (p.variant != 0) return "plan variant must be 0";
  if (tier == RSIM_TIER_FP32) {
    if (p.tile_n != 0 && p.tile_n != 64 && p.tile_n != 128) return "FP32 tile_n must be 64 or 128";
  } else if (tensor_tier(tier)) {
    const int lmax = std::max(8, (k.L + 7) / 8 * 8);
    if (p.tile_n != 0 && (p.tile_n < 8 || p.tile_n > 128 || p.tile_n % 8 != 0 || p.tile_n > lmax))
      return "tensor-core tile_n must be a multiple of 8 in 8..min(128, L rounded up to 8)";
    if (p.group_chunks < 0 || p.group_chunks > group_chunks_max(tier))
      return "group_chunks must be in 1.." + std::to_string(group_chunks_max(tier)) + " for this tier";
  }
  return std::string();
}

}  // namespace rsim
