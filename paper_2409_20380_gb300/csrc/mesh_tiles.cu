// Host-side construction of the hex-patch tiling used by the tiled EBE kernel.
//
// A mesh qualifies when its elements come in groups of six consecutive tetrahedra that cover the eight
// corners of a hexahedron with one fixed local topology (the Kuhn split: every tet contains the two
// corners of one main diagonal).  The geometry of each tet stays general; only the topology is shared.
// Slots are numbered by first appearance when scanning a group's six tets node by node, so the whole
// topology is the table kHexTet below.  Consecutive runs of `hex_per_tile` hexes form a tile; a tile
// lists its distinct nodes (flagged when another tile also touches them) and, per hex, the tile-local
// index of each of its eight corners.
#include <algorithm>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

bool detect_hex_patches(const int32_t* conn, int64_t E) {
  if (E % 6 != 0 || E == 0) return false;
  const int64_t H = E / 6;
  for (int64_t h = 0; h < H; ++h) {
    int nodes[8];
    int n = 0;
    for (int t = 0; t < 6; ++t)
      for (int a = 0; a < 4; ++a) {
        const int id = conn[(h * 6 + t) * 4 + a];
        int slot = -1;
        for (int s = 0; s < n; ++s)
          if (nodes[s] == id) slot = s;
        if (slot < 0) {
          if (n == 8) return false;
          nodes[n] = id;
          slot = n++;
        }
        if (slot != kHexTet[t][a]) return false;
      }
    if (n != 8) return false;
  }
  return true;
}

bool build_hex_tiles(const int32_t* conn, int64_t E, int64_t N, int hex_per_tile, HexTilesHost* out) {
  const int64_t H = E / 6;
  out->hex_per_tile = hex_per_tile;
  out->n_hex = H;
  const int64_t n_tiles = (H + hex_per_tile - 1) / hex_per_tile;
  out->n_tiles = (int)n_tiles;
  std::vector<int> hex_count(N, 0);      // hexes touching each node
  // corner s of hex h: the node that first appears at slot s
  auto corner = [&](int64_t h, int s) -> int {
    for (int t = 0; t < 6; ++t)
      for (int a = 0; a < 4; ++a)
        if (kHexTet[t][a] == s) return conn[(h * 6 + t) * 4 + a];
    return -1;
  };
  std::vector<int> corners((size_t)H * 8);
  for (int64_t h = 0; h < H; ++h)
    for (int s = 0; s < 8; ++s) {
      const int id = corner(h, s);
      corners[h * 8 + s] = id;
      hex_count[id] += 1;
    }
  out->tile_hex_off.assign(n_tiles + 1, 0);
  out->tile_node_off.assign(n_tiles + 1, 0);
  out->tile_nodes.clear();
  out->hex_local.assign((size_t)H * 8, 0);
  out->nloc_max = 0;
  std::vector<int> loc;
  std::vector<int> tcount;
  for (int64_t t = 0; t < n_tiles; ++t) {
    const int64_t h0 = t * hex_per_tile, h1 = std::min<int64_t>(H, h0 + hex_per_tile);
    out->tile_hex_off[t] = (int)h0;
    loc.assign(corners.begin() + h0 * 8, corners.begin() + h1 * 8);
    std::sort(loc.begin(), loc.end());
    loc.erase(std::unique(loc.begin(), loc.end()), loc.end());
    if (loc.size() > 65535) return false;
    tcount.assign(loc.size(), 0);
    for (int64_t h = h0; h < h1; ++h)
      for (int s = 0; s < 8; ++s) {
        const int l = (int)(std::lower_bound(loc.begin(), loc.end(), corners[h * 8 + s]) - loc.begin());
        out->hex_local[h * 8 + s] = (uint16_t)l;
        tcount[l] += 1;
      }
    out->tile_node_off[t] = (int)out->tile_nodes.size();
    for (size_t l = 0; l < loc.size(); ++l) {
      const bool shared = tcount[l] < hex_count[loc[l]];
      out->tile_nodes.push_back(shared ? (int)(loc[l] | 0x80000000u) : loc[l]);
    }
    out->nloc_max = std::max(out->nloc_max, (int)loc.size());
  }
  out->tile_hex_off[n_tiles] = (int)H;
  out->tile_node_off[n_tiles] = (int)out->tile_nodes.size();
  return true;
}

}  // namespace fem
