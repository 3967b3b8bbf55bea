// Conforming unstructured hexahedral meshes (host code): the numbering of the order-p H1
// degrees of freedom -- the global (L-vector) level of Fig. "fig_feod", Sec. 3.5 -- and the
// element -> DOF map G built from the element connectivity alone.
//
// An element lists its 8 vertices in the tensor-product corner order: corner (i, j, k) of the
// reference cube [0,1]^3 is entry i + 2j + 4k.  Its local nodes are the (p+1)^3 GLL points
// (a, b, c), a fastest.  A node lies on a vertex, on the interior of an edge or a face, or in the
// element's interior.  Edge and face nodes are shared between the elements that hold that
// edge or face, so they need a frame every element agrees on:
//   - edge: its p-1 nodes are counted from the end with the smaller global vertex id;
//   - face: its (p-1)^2 nodes are indexed in a frame whose origin is the face's vertex with the
//     smallest global id and whose first axis points to the smaller-id of that vertex's two
//     neighbours on the face (the GLL nodes are symmetric about 1/2, so node t from one end is
//     node p - t from the other).
// Global numbers are handed out entity by entity in the order the elements first touch them
// (elements in the given order, nodes in local order), which keeps each element's DOFs close
// together when the element order has locality.
#pragma once

#include <algorithm>
#include <array>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

namespace fepa {
namespace hexmesh {

struct Numbering {
  int64_t ndofs = 0;
  std::vector<int32_t> gmap;      // [E][(p+1)^3] global DOF of each element-local node
  std::vector<int32_t> boundary;  // DOFs on the faces that belong to one element only, ascending
  std::string error;              // reason when number_dofs returns false
};

// the 12 edges: free direction d, the fixed bits of the other two directions (lower one first)
struct LocalEdge { int d, lo_dir, hi_dir, lo_bit, hi_bit; };
// the 6 faces: fixed direction d0 at value f; free directions d1 < d2
struct LocalFace { int d0, f, d1, d2; };

inline int corner(const int bits[3]) { return bits[0] + 2 * bits[1] + 4 * bits[2]; }

inline std::array<LocalEdge, 12> local_edges() {
  std::array<LocalEdge, 12> out{};
  int k = 0;
  for (int d = 0; d < 3; ++d) {
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    for (int b2 = 0; b2 < 2; ++b2)
      for (int b1 = 0; b1 < 2; ++b1) out[k++] = {d, o1, o2, b1, b2};
  }
  return out;
}

inline std::array<LocalFace, 6> local_faces() {
  std::array<LocalFace, 6> out{};
  int k = 0;
  for (int d0 = 0; d0 < 3; ++d0)
    for (int f = 0; f < 2; ++f) out[k++] = {d0, f, d0 == 0 ? 1 : 0, d0 == 2 ? 1 : 2};
  return out;
}

// global vertex ids of a local face, FV[u][w] = corner with d0 = f, d1 = u, d2 = w
inline void face_vertices(const int32_t* cv, const LocalFace& lf, int32_t FV[2][2]) {
  for (int u = 0; u < 2; ++u)
    for (int w = 0; w < 2; ++w) {
      int bits[3];
      bits[lf.d0] = lf.f;
      bits[lf.d1] = u;
      bits[lf.d2] = w;
      FV[u][w] = cv[corner(bits)];
    }
}

struct FaceKey {
  std::array<int32_t, 4> v;  // sorted vertex ids
  bool operator==(const FaceKey& o) const { return v == o.v; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t x : k.v) h = (h ^ (uint64_t)(uint32_t)x) * 1099511628211ull;
    return (size_t)h;
  }
};
struct FaceRec {
  int64_t base = -1;        // first DOF of the face's interior nodes
  int count = 0;            // elements holding the face
  int64_t elem = -1;        // first element holding it, and its local face
  int lface = -1;
  std::pair<int32_t, int32_t> diag{-1, -1};  // one diagonal (sorted ids), to check the faces match
};

inline FaceKey face_key(const int32_t FV[2][2]) {
  FaceKey k{{FV[0][0], FV[1][0], FV[0][1], FV[1][1]}};
  std::sort(k.v.begin(), k.v.end());
  return k;
}

inline std::pair<int32_t, int32_t> face_diag(const int32_t FV[2][2]) {
  return {std::min(FV[0][0], FV[1][1]), std::max(FV[0][0], FV[1][1])};
}

// Numbers the DOFs of order p on the mesh (nverts vertices, E elements, conn [E][8]).
// Fails (returns false with out.error set) on vertex ids out of range, an element with a
// repeated vertex, a face held by more than two elements, two elements whose common four
// vertices form different quadrilaterals, or more DOFs than 32-bit flagged indices allow.
inline bool number_dofs(int64_t nverts, int64_t E, const int32_t* conn, int p, Numbering& out,
                        int64_t max_dofs = (int64_t)1 << 30) {
  out = Numbering();
  const int n = p + 1, m = p - 1;
  const int64_t n3 = (int64_t)n * n * n;
  if (p < 1) { out.error = "order must be >= 1"; return false; }
  if (E < 1 || nverts < 1) { out.error = "need at least one element and one vertex"; return false; }
  if (E * n3 >= ((int64_t)1 << 31)) { out.error = "too many element-local nodes for 32-bit indices"; return false; }
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* cv = conn + 8 * e;
    for (int c = 0; c < 8; ++c) {
      if (cv[c] < 0 || cv[c] >= nverts) {
        out.error = "element " + std::to_string(e) + ": vertex id out of range";
        return false;
      }
      for (int c2 = 0; c2 < c; ++c2)
        if (cv[c2] == cv[c]) {
          out.error = "element " + std::to_string(e) + ": repeated vertex";
          return false;
        }
    }
  }
  const auto LE = local_edges();
  const auto LF = local_faces();

  // faces: multiplicity and matching
  std::unordered_map<FaceKey, FaceRec, FaceKeyHash> faces;
  faces.reserve((size_t)(3 * E + 16));
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* cv = conn + 8 * e;
    for (int f = 0; f < 6; ++f) {
      int32_t FV[2][2];
      face_vertices(cv, LF[f], FV);
      FaceRec& r = faces[face_key(FV)];
      if (r.count == 0) {
        r.elem = e;
        r.lface = f;
        r.diag = face_diag(FV);
      } else {
        const auto dg = face_diag(FV);
        const std::pair<int32_t, int32_t> other = {std::min(FV[1][0], FV[0][1]), std::max(FV[1][0], FV[0][1])};
        if (dg != r.diag && other != r.diag) {
          out.error = "element " + std::to_string(e) + ": a face's four vertices form a different quadrilateral "
                      "in a neighbouring element";
          return false;
        }
      }
      if (++r.count > 2) {
        out.error = "element " + std::to_string(e) + ": a face is held by more than two elements";
        return false;
      }
    }
  }

  std::vector<int64_t> vdof((size_t)nverts, -1);
  std::unordered_map<uint64_t, int64_t> edge_base;
  edge_base.reserve((size_t)(4 * E + 16));
  int64_t next = 0;
  out.gmap.resize((size_t)(E * n3));
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* cv = conn + 8 * e;
    // bases and orientation of this element's 12 edges and 6 faces
    int64_t eb[12];
    bool eflip[12];
    for (int k = 0; k < 12; ++k) {
      const LocalEdge& le = LE[k];
      int ba[3], bb[3];
      ba[le.d] = 0;
      bb[le.d] = 1;
      ba[le.lo_dir] = bb[le.lo_dir] = le.lo_bit;
      ba[le.hi_dir] = bb[le.hi_dir] = le.hi_bit;
      const int32_t va = cv[corner(ba)], vb = cv[corner(bb)];
      eflip[k] = va > vb;  // local direction runs from the larger id
      if (m > 0) {
        const uint64_t key = ((uint64_t)(uint32_t)std::min(va, vb) << 32) | (uint32_t)std::max(va, vb);
        auto it = edge_base.find(key);
        if (it == edge_base.end()) {
          it = edge_base.emplace(key, next).first;
          next += m;
        }
        eb[k] = it->second;
      }
    }
    int64_t fb[6];
    int fu0[6], fw0[6];
    bool fswap[6];
    for (int f = 0; f < 6; ++f) {
      int32_t FV[2][2];
      face_vertices(cv, LF[f], FV);
      int u0 = 0, w0 = 0;
      for (int u = 0; u < 2; ++u)
        for (int w = 0; w < 2; ++w)
          if (FV[u][w] < FV[u0][w0]) { u0 = u; w0 = w; }
      fu0[f] = u0;
      fw0[f] = w0;
      fswap[f] = FV[u0][1 - w0] < FV[1 - u0][w0];  // first canonical axis along d2
      if (m > 0) {
        FaceRec& r = faces[face_key(FV)];
        if (r.base < 0) {
          r.base = next;
          next += (int64_t)m * m;
        }
        fb[f] = r.base;
      }
    }
    int64_t ib = -1;
    for (int64_t l = 0; l < n3; ++l) {
      const int idx[3] = {(int)(l % n), (int)((l / n) % n), (int)(l / ((int64_t)n * n))};
      int onb = 0;
      for (int d = 0; d < 3; ++d) onb += (idx[d] == 0 || idx[d] == p);
      int64_t g;
      if (onb == 3) {
        const int bits[3] = {idx[0] / p, idx[1] / p, idx[2] / p};
        const int32_t v = cv[corner(bits)];
        if (vdof[v] < 0) vdof[v] = next++;
        g = vdof[v];
      } else if (onb == 2) {
        int d = 0;
        while (idx[d] == 0 || idx[d] == p) ++d;
        int k = 0;
        for (; k < 12; ++k) {
          const LocalEdge& le = LE[k];
          if (le.d == d && idx[le.lo_dir] == le.lo_bit * p && idx[le.hi_dir] == le.hi_bit * p) break;
        }
        const int t = idx[d];
        g = eb[k] + (eflip[k] ? (p - t) - 1 : t - 1);
      } else if (onb == 1) {
        int d0 = 0;
        while (!(idx[d0] == 0 || idx[d0] == p)) ++d0;
        const int f = 2 * d0 + idx[d0] / p;
        const LocalFace& lf = LF[f];
        const int r1 = fu0[f] ? p - idx[lf.d1] : idx[lf.d1];
        const int r2 = fw0[f] ? p - idx[lf.d2] : idx[lf.d2];
        const int s1 = fswap[f] ? r2 : r1, s2 = fswap[f] ? r1 : r2;
        g = fb[f] + (s1 - 1) + (int64_t)m * (s2 - 1);
      } else {
        if (ib < 0) {
          ib = next;
          next += (int64_t)m * m * m;
        }
        g = ib + (idx[0] - 1) + (int64_t)m * ((idx[1] - 1) + (int64_t)m * (idx[2] - 1));
      }
      if (next > max_dofs) {
        out.error = "too many DOFs for 32-bit flagged indices";
        return false;
      }
      out.gmap[(size_t)(e * n3 + l)] = (int32_t)g;
    }
  }
  out.ndofs = next;

  // boundary: every node of a face that one element holds
  std::vector<char> on((size_t)next, 0);
  for (const auto& kv : faces) {
    const FaceRec& r = kv.second;
    if (r.count != 1) continue;
    const LocalFace& lf = LF[r.lface];
    for (int64_t l = 0; l < n3; ++l) {
      const int idx[3] = {(int)(l % n), (int)((l / n) % n), (int)(l / ((int64_t)n * n))};
      if (idx[lf.d0] == lf.f * p) on[(size_t)out.gmap[(size_t)(r.elem * n3 + l)]] = 1;
    }
  }
  for (int64_t g = 0; g < next; ++g)
    if (on[(size_t)g]) out.boundary.push_back((int32_t)g);
  return true;
}

}  // namespace hexmesh
}  // namespace fepa
