// Q_p connectivity of an unstructured hexahedral mesh given only by its
// elements' vertices (the paper's unstructured setting, sections "Benchmarks"
// and "libCEED": the element restriction G maps global nodes to element-local
// ones).  Host code; the result feeds fem_mesh_create*.
//
// Numbering: every node of the Q_p space belongs to one mesh entity --
// vertex, edge, face or element interior -- and entities shared by elements
// whose local frames differ must give each shared node one global id:
//   vertex    the vertex itself;
//   edge      p-1 nodes ordered from the edge's lower global vertex;
//   face      (p-1)^2 nodes in a canonical frame: origin at the face's lowest
//             global vertex, first axis towards the lower of that corner's
//             two face neighbours;
//   interior  (p-1)^3 nodes of the element alone.
// Global ids are assigned in order of first use (elements in order, local
// nodes a + P b + P^2 c), so a lexicographic mesh keeps its locality.
// Dirichlet nodes: every node of a face that belongs to one element only.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <unordered_map>
#include <vector>

#include "fem_internal.h"

namespace {

struct FaceKey {
  std::array<int32_t, 4> v;
  bool operator==(const FaceKey &o) const { return v == o.v; }
};
struct FaceHash {
  size_t operator()(const FaceKey &k) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t x : k.v) { h ^= (uint64_t)(uint32_t)x; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

struct FaceInfo {
  int64_t base = -1;   // first global id of the (p-1)^2 interior nodes
  int count = 0;       // elements that share the face
};

}  // namespace

extern "C" fem_status fem_mesh_connectivity(int p, int64_t nvert, int64_t E, const int32_t *elem_verts,
                                            int32_t *elem_nodes, uint8_t *dirichlet, int64_t *N_out) {
  if (p < 1 || p + 1 > FEM_MAX_P || nvert < 1 || E < 1 || !elem_verts || !elem_nodes || !N_out) {
    fem_set_error("fem_mesh_connectivity: invalid arguments (p=%d, nvert=%lld, E=%lld)", p,
                  (long long)nvert, (long long)E);
    return FEM_EINVAL;
  }
  const int P = p + 1, P3 = P * P * P, pm = p - 1;
  if ((int64_t)E * P3 > INT32_MAX) {
    fem_set_error("fem_mesh_connectivity: E * (p+1)^3 exceeds the int32 node index range");
    return FEM_EINVAL;
  }
  for (int64_t e = 0; e < E; e++) {
    const int32_t *ev = elem_verts + 8 * e;
    for (int a = 0; a < 8; a++) {
      if (ev[a] < 0 || ev[a] >= nvert) {
        fem_set_error("fem_mesh_connectivity: element %lld vertex %d out of range", (long long)e, a);
        return FEM_EINVAL;
      }
      for (int b = 0; b < a; b++)
        if (ev[a] == ev[b]) {
          fem_set_error("fem_mesh_connectivity: element %lld repeats vertex %d", (long long)e, ev[a]);
          return FEM_EINVAL;
        }
    }
  }
  std::vector<int64_t> vid(nvert, -1);
  std::unordered_map<uint64_t, int64_t> edges;   // (lo, hi) -> first id
  std::unordered_map<FaceKey, FaceInfo, FaceHash> faces;
  edges.reserve((size_t)E * 3);
  faces.reserve((size_t)E * 3);
  int64_t next = 0;
  auto local_vertex = [](int i, int j, int k) { return i + 2 * j + 4 * k; };
  // the 6 local faces: fixed direction d at side s (0 or p)
  for (int64_t e = 0; e < E; e++) {
    const int32_t *ev = elem_verts + 8 * e;
    int32_t *en = elem_nodes + e * P3;
    for (int c = 0; c < P; c++)
      for (int b = 0; b < P; b++)
        for (int a = 0; a < P; a++) {
          const int crd[3] = {a, b, c};
          int onb = 0;
          for (int d = 0; d < 3; d++) onb += (crd[d] == 0 || crd[d] == p);
          int64_t id;
          if (onb == 3) {                                   // vertex
            const int32_t g = ev[local_vertex(a / p, b / p, c / p)];
            if (vid[g] < 0) vid[g] = next++;
            id = vid[g];
          } else if (onb == 2) {                            // edge
            int d = 0;
            while (crd[d] == 0 || crd[d] == p) d++;
            int lo[3] = {a / p, b / p, c / p}, hi[3] = {a / p, b / p, c / p};
            lo[d] = 0; hi[d] = 1;
            const int32_t gA = ev[local_vertex(lo[0], lo[1], lo[2])];
            const int32_t gB = ev[local_vertex(hi[0], hi[1], hi[2])];
            const uint64_t key = ((uint64_t)(uint32_t)std::min(gA, gB) << 32) | (uint32_t)std::max(gA, gB);
            auto it = edges.find(key);
            int64_t base;
            if (it == edges.end()) { base = next; next += pm; edges.emplace(key, base); }
            else base = it->second;
            const int t = crd[d];                           // 1..p-1 from A
            id = base + (gA < gB ? t - 1 : pm - t);
          } else if (onb == 1) {                            // face
            int d = 0;
            while (!(crd[d] == 0 || crd[d] == p)) d++;
            const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;   // free directions, ascending
            int32_t G[2][2];
            for (int w0 = 0; w0 < 2; w0++)
              for (int u0 = 0; u0 < 2; u0++) {
                int v[3];
                v[d] = crd[d] / p; v[d1] = u0; v[d2] = w0;
                G[u0][w0] = ev[local_vertex(v[0], v[1], v[2])];
              }
            FaceKey key{{G[0][0], G[1][0], G[0][1], G[1][1]}};
            std::sort(key.v.begin(), key.v.end());
            // canonical frame: corner with the lowest id, first axis towards
            // its lower face neighbour
            int cu = 0, cw = 0;
            for (int w0 = 0; w0 < 2; w0++)
              for (int u0 = 0; u0 < 2; u0++)
                if (G[u0][w0] < G[cu][cw]) { cu = u0; cw = w0; }
            const bool along_u = G[1 - cu][cw] < G[cu][1 - cw];
            const int u = crd[d1], w = crd[d2];
            const int du = cu ? p - u : u, dw = cw ? p - w : w;   // distances from the corner
            const int s = along_u ? du : dw, t = along_u ? dw : du;
            FaceInfo &fi = faces[key];
            if (fi.base < 0) { fi.base = next; next += (int64_t)pm * pm; }
            id = fi.base + (s - 1) + (int64_t)pm * (t - 1);
          } else {                                          // interior
            id = -1;   // numbered below, after the element's shared nodes
          }
          en[a + P * (b + P * c)] = (int32_t)id;
        }
    // interior nodes in local order
    for (int c = 1; c < p; c++)
      for (int b = 1; b < p; b++)
        for (int a = 1; a < p; a++) en[a + P * (b + P * c)] = (int32_t)(next++);
    // face use counts (once per element face)
    for (int d = 0; d < 3; d++)
      for (int side = 0; side < 2; side++) {
        const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
        FaceKey key;
        int m = 0;
        for (int w0 = 0; w0 < 2; w0++)
          for (int u0 = 0; u0 < 2; u0++) {
            int v[3];
            v[d] = side; v[d1] = u0; v[d2] = w0;
            key.v[m++] = ev[local_vertex(v[0], v[1], v[2])];
          }
        std::sort(key.v.begin(), key.v.end());
        FaceInfo &fi = faces[key];
        fi.count += 1;
        if (fi.count > 2) {
          fem_set_error("fem_mesh_connectivity: a face of element %lld is shared by more than two elements",
                        (long long)e);
          return FEM_EINVAL;
        }
      }
  }
  if (next > INT32_MAX) {
    fem_set_error("fem_mesh_connectivity: %lld nodes exceed the int32 index range", (long long)next);
    return FEM_EINVAL;
  }
  *N_out = next;
  if (dirichlet) {
    memset(dirichlet, 0, (size_t)next);
    for (int64_t e = 0; e < E; e++) {
      const int32_t *ev = elem_verts + 8 * e;
      const int32_t *en = elem_nodes + e * P3;
      for (int d = 0; d < 3; d++)
        for (int side = 0; side < 2; side++) {
          const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
          FaceKey key;
          int m = 0;
          for (int w0 = 0; w0 < 2; w0++)
            for (int u0 = 0; u0 < 2; u0++) {
              int v[3];
              v[d] = side; v[d1] = u0; v[d2] = w0;
              key.v[m++] = ev[local_vertex(v[0], v[1], v[2])];
            }
          std::sort(key.v.begin(), key.v.end());
          if (faces[key].count != 1) continue;
          for (int w = 0; w < P; w++)
            for (int u = 0; u < P; u++) {
              int crd[3];
              crd[d] = side * p; crd[d1] = u; crd[d2] = w;
              dirichlet[en[crd[0] + P * (crd[1] + P * crd[2])]] = 1;
            }
        }
    }
  }
  return FEM_OK;
}
