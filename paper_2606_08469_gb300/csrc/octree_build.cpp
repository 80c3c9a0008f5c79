// Host octree builder: seeded adaptive octree (or one from explicit split
// flags) flattened into level-ordered arrays.  The paper builds its sparse
// multi-level octree from the scene geometry (Section 3.4, Section 4.1); the
// seeded generator stands in for it.
#include <cstring>
#include <vector>

#include "octa_internal.h"

namespace {

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), from its published
// definition: golden-gamma increment, then the 30/27/31 xor-shift-multiply
// finaliser.
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double unit() { return static_cast<double>(next() >> 11) * 0x1.0p-53; }
};

constexpr int64_t kMaxCount = 2147483647;  // int32 indices in the flat arrays

// Breadth-first construction; decide(depth) is called once for every node
// whose depth is below max_depth, in node order.
template <class Decide>
int bfs_build(Decide&& decide, int32_t max_depth, const int32_t* R, octa_tree_desc* desc,
              int32_t* first_child, int32_t* node_coord, int32_t* map_offset) {
  if (!desc || !R) return octa::fail(OCTA_EINVAL, "octree: desc and R must be non-NULL");
  if (max_depth < 0 || max_depth >= OCTA_MAX_LEVELS)
    return octa::fail(OCTA_ERANGE, "octree: max_depth %d outside [0, %d]", max_depth,
                      OCTA_MAX_LEVELS - 1);
  const int K = max_depth + 1;
  for (int l = 0; l < K; ++l)
    if (R[l] < 2 || R[l] > 4096)
      return octa::fail(OCTA_ERANGE, "octree: R[%d] = %d outside [2, 4096]", l, R[l]);

  std::vector<int32_t> fc;
  std::vector<int32_t> coord{0, 0, 0};
  std::vector<int8_t> level{0};
  for (size_t i = 0; i < level.size(); ++i) {
    const int d = level[i];
    if (d < max_depth && decide(d)) {
      if (static_cast<int64_t>(level.size()) + 8 > kMaxCount)
        return octa::fail(OCTA_ERANGE, "octree: more than 2^31-1 nodes");
      fc.push_back(static_cast<int32_t>(level.size()));
      const int32_t cx = coord[3 * i], cy = coord[3 * i + 1], cz = coord[3 * i + 2];
      for (int b = 0; b < 8; ++b) {
        coord.push_back(2 * cx + (b & 1));
        coord.push_back(2 * cy + ((b >> 1) & 1));
        coord.push_back(2 * cz + ((b >> 2) & 1));
        level.push_back(static_cast<int8_t>(d + 1));
      }
    } else {
      fc.push_back(-1);
    }
  }
  const int64_t n = static_cast<int64_t>(level.size());
  octa_tree_desc out;
  std::memset(&out, 0, sizeof(out));
  out.num_levels = K;
  out.num_nodes = static_cast<int32_t>(n);
  for (int l = 0; l < K; ++l) out.R[l] = R[l];
  // levels are contiguous in breadth-first order
  int64_t i = 0;
  for (int l = 0; l <= K; ++l) {
    while (i < n && level[i] < l) ++i;
    out.level_node_start[l] = static_cast<int32_t>(i);
  }
  out.level_node_start[K] = static_cast<int32_t>(n);
  out.level_texel_base[0] = 0;
  for (int l = 0; l < K; ++l) {
    const int64_t cnt = out.level_node_start[l + 1] - out.level_node_start[l];
    out.level_texel_base[l + 1] = out.level_texel_base[l] + cnt * R[l] * R[l];
  }
  out.num_texels = out.level_texel_base[K];
  if (out.num_texels > kMaxCount)
    return octa::fail(OCTA_ERANGE, "octree: %lld texels exceed 2^31-1",
                      static_cast<long long>(out.num_texels));
  *desc = out;
  if (!first_child) return OCTA_OK;  // sizing call
  if (!node_coord || !map_offset)
    return octa::fail(OCTA_EINVAL, "octree: node_coord and map_offset must be non-NULL");
  for (int64_t k = 0; k < n; ++k) {
    first_child[k] = fc[k];
    for (int c = 0; c < 3; ++c) node_coord[3 * k + c] = coord[3 * k + c];
    const int l = level[k];
    map_offset[k] = static_cast<int32_t>(out.level_texel_base[l] +
                                         (k - out.level_node_start[l]) * R[l] * R[l]);
  }
  return OCTA_OK;
}

}  // namespace

extern "C" int octree_build(uint64_t seed, int32_t max_depth, double p_base, const int32_t* R,
                            octa_tree_desc* desc, int32_t* first_child, int32_t* node_coord,
                            int32_t* map_offset) {
  octa::clear_error();
  if (!(p_base >= 0.0 && p_base <= 1.0))
    return octa::fail(OCTA_EINVAL, "octree_build: p_base must lie in [0, 1]");
  if (max_depth < 0 || max_depth >= OCTA_MAX_LEVELS)
    return octa::fail(OCTA_ERANGE, "octree_build: max_depth %d outside [0, %d]", max_depth,
                      OCTA_MAX_LEVELS - 1);
  double thr[OCTA_MAX_LEVELS];
  thr[0] = 1.0;
  for (int d = 1; d < OCTA_MAX_LEVELS; ++d) thr[d] = thr[d - 1] * p_base;
  SplitMix64 rng{seed};
  return bfs_build([&](int d) { return rng.unit() < thr[d]; }, max_depth, R, desc, first_child,
                   node_coord, map_offset);
}

extern "C" int octree_from_flags(const uint8_t* flags, int64_t n_flags, int32_t max_depth,
                                 const int32_t* R, octa_tree_desc* desc, int32_t* first_child,
                                 int32_t* node_coord, int32_t* map_offset) {
  octa::clear_error();
  if (n_flags < 0 || (n_flags > 0 && !flags))
    return octa::fail(OCTA_EINVAL, "octree_from_flags: flags NULL with n_flags > 0");
  int64_t k = 0;
  return bfs_build(
      [&](int) {
        const int64_t j = k++;
        return j < n_flags && flags[j] != 0;
      },
      max_depth, R, desc, first_child, node_coord, map_offset);
}
