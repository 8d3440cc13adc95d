// Box partition of a structured hexahedral mesh over ranks (host, no GPU):
// the layout a sharded solve would use, and the exchange lists that make the
// distributed sums of the path identical to the single-domain ones.
//
// Ranks form a px x py x pz grid; rank r owns a box of cells (balanced split
// per axis) and holds the GLL nodes of its cells (its node box, shared with
// neighbours on the box faces, edges and corners).  A stiffness apply or the
// scatter of the relaxation produces per-cell contributions E[cell][node];
// the value at a node is their sum over the cells that contain it, which the
// single-domain node gather forms in ascending global cell index.  Here each
// rank sends, to each neighbour, its own cells' contributions at the nodes
// the two node boxes share (nodes ascending, then cells ascending) and sums
// every node of its box with a plan that lists the contributions in ascending
// global cell index, own (local E index) or received (receive-buffer slot):
// the result equals the single-domain sum bit for bit.  A node has one owner
// (the box whose half-open cell range contains the node's lower cell along
// every axis, the last box for the upper boundary), which takes it in dot
// products; a vertex star belongs to the owner of its vertex, whose cells plus
// a one-cell halo contain all of the star's cells.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fdmpc.h"

namespace {

struct Axis {
  int n = 0, P = 0;  // cells, ranks along the axis
  int c0(int r) const { return (int)(((int64_t)r * n) / P); }
  int c1(int r) const { return (int)(((int64_t)(r + 1) * n) / P); }
  int rank_of_cell(int c) const {  // the r with c0(r) <= c < c1(r)
    int r = (int)(((int64_t)c * P) / n);
    while (r > 0 && c < c0(r)) --r;
    while (r < P - 1 && c >= c1(r)) ++r;
    return r;
  }
};

}  // namespace

struct fdm_partition {
  int p = 0, n = 0;
  Axis ax[3];
  int rc[3] = {0, 0, 0};  // this rank's coordinates in the rank grid
  int rank = 0;
  int cb[6] = {0};        // owned cells [c0, c1) per axis
  int nb[6] = {0};        // node box [g0, g1] per axis (inclusive)
  int hb[6] = {0};        // cells with the one-cell halo [c0, c1) per axis
  std::vector<int> neigh;
  std::vector<int64_t> send_ptr, send, recv_ptr, sum_ptr, sum;
  std::vector<uint8_t> owned;
  std::vector<int64_t> stars;  // global vertex indices of the stars this rank owns
  std::string err;
};

namespace {

thread_local std::string g_part_err;

int rank_id(const fdm_partition *P, const int c[3]) { return c[0] + P->ax[0].P * (c[1] + P->ax[1].P * c[2]); }

// cells containing node coordinate g along an axis with nc cells (ascending)
int cells_of(int g, int p, int nc, int out[2]) {
  const int q = g / p;
  int k = 0;
  if (g % p == 0) {
    if (q - 1 >= 0) out[k++] = q - 1;
    if (q < nc) out[k++] = q;
  } else {
    out[k++] = q;
  }
  return k;
}

void build(fdm_partition *P) {
  const int p = P->p, n = P->n, n3 = n * n * n;
  for (int a = 0; a < 3; ++a) {
    const Axis &A = P->ax[a];
    P->cb[2 * a] = A.c0(P->rc[a]);
    P->cb[2 * a + 1] = A.c1(P->rc[a]);
    P->nb[2 * a] = P->cb[2 * a] * p;
    P->nb[2 * a + 1] = P->cb[2 * a + 1] * p;
    P->hb[2 * a] = std::max(0, P->cb[2 * a] - 1);
    P->hb[2 * a + 1] = std::min(A.n, P->cb[2 * a + 1] + 1);
  }
  const int w[3] = {P->cb[1] - P->cb[0], P->cb[3] - P->cb[2], P->cb[5] - P->cb[4]};
  const int N[3] = {P->ax[0].n * p + 1, P->ax[1].n * p + 1, P->ax[2].n * p + 1};
  auto own_cell = [&](const int c[3]) {
    for (int a = 0; a < 3; ++a)
      if (c[a] < P->cb[2 * a] || c[a] >= P->cb[2 * a + 1]) return false;
    return true;
  };
  auto local_e = [&](const int c[3], const int g[3]) -> int64_t {
    const int64_t lc = (c[0] - P->cb[0]) + (int64_t)w[0] * ((c[1] - P->cb[2]) + (int64_t)w[1] * (c[2] - P->cb[4]));
    const int l = (g[0] - c[0] * p) + n * ((g[1] - c[1] * p) + n * (g[2] - c[2] * p));
    return lc * n3 + l;
  };
  // neighbours: every other rank whose node box meets this one (ascending rank)
  std::vector<std::array<int, 6>> boxes;
  for (int rz = 0; rz < P->ax[2].P; ++rz)
    for (int ry = 0; ry < P->ax[1].P; ++ry)
      for (int rx = 0; rx < P->ax[0].P; ++rx) {
        const int r[3] = {rx, ry, rz};
        const int id = rank_id(P, r);
        if (id == P->rank) continue;
        std::array<int, 6> is;
        bool meet = true;
        for (int a = 0; a < 3; ++a) {
          const int g0 = P->ax[a].c0(r[a]) * p, g1 = P->ax[a].c1(r[a]) * p;
          is[2 * a] = std::max(g0, P->nb[2 * a]);
          is[2 * a + 1] = std::min(g1, P->nb[2 * a + 1]);
          meet = meet && is[2 * a] <= is[2 * a + 1];
        }
        if (!meet) continue;
        P->neigh.push_back(id);
        boxes.push_back(is);
      }
  // send and receive lists per neighbour; receive slots keyed by (node, cell)
  std::map<std::pair<int64_t, int64_t>, int64_t> slot;
  P->send_ptr.assign(1, 0);
  P->recv_ptr.assign(1, 0);
  int64_t nrecv = 0;
  for (size_t k = 0; k < P->neigh.size(); ++k) {
    const std::array<int, 6> &is = boxes[k];
    for (int gz = is[4]; gz <= is[5]; ++gz)
      for (int gy = is[2]; gy <= is[3]; ++gy)
        for (int gx = is[0]; gx <= is[1]; ++gx) {
          const int g[3] = {gx, gy, gz};
          const int64_t gid = gx + (int64_t)N[0] * (gy + (int64_t)N[1] * gz);
          int cl[3][2], cn[3];
          for (int a = 0; a < 3; ++a) cn[a] = cells_of(g[a], p, P->ax[a].n, cl[a]);
          for (int iz = 0; iz < cn[2]; ++iz)
            for (int iy = 0; iy < cn[1]; ++iy)
              for (int ix = 0; ix < cn[0]; ++ix) {
                const int c[3] = {cl[0][ix], cl[1][iy], cl[2][iz]};
                const int rr[3] = {P->ax[0].rank_of_cell(c[0]), P->ax[1].rank_of_cell(c[1]), P->ax[2].rank_of_cell(c[2])};
                const int owner = rank_id(P, rr);
                const int64_t cid = c[0] + (int64_t)P->ax[0].n * (c[1] + (int64_t)P->ax[1].n * c[2]);
                if (owner == P->rank) P->send.push_back(local_e(c, g));
                else if (owner == P->neigh[k]) slot[{gid, cid}] = nrecv++;
              }
        }
    P->send_ptr.push_back((int64_t)P->send.size());
    P->recv_ptr.push_back(nrecv);
  }
  // the sum plan of every node of the node box (x fastest), and ownership
  const int L[3] = {P->nb[1] - P->nb[0] + 1, P->nb[3] - P->nb[2] + 1, P->nb[5] - P->nb[4] + 1};
  P->sum_ptr.assign(1, 0);
  P->owned.resize((size_t)L[0] * L[1] * L[2]);
  size_t li = 0;
  for (int gz = P->nb[4]; gz <= P->nb[5]; ++gz)
    for (int gy = P->nb[2]; gy <= P->nb[3]; ++gy)
      for (int gx = P->nb[0]; gx <= P->nb[1]; ++gx, ++li) {
        const int g[3] = {gx, gy, gz};
        const int64_t gid = gx + (int64_t)N[0] * (gy + (int64_t)N[1] * gz);
        int cl[3][2], cn[3];
        bool own = true;
        for (int a = 0; a < 3; ++a) {
          cn[a] = cells_of(g[a], p, P->ax[a].n, cl[a]);
          const int lowc = std::min(g[a] / p, P->ax[a].n - 1);
          own = own && P->ax[a].rank_of_cell(lowc) == P->rc[a];
        }
        P->owned[li] = own ? 1 : 0;
        for (int iz = 0; iz < cn[2]; ++iz)
          for (int iy = 0; iy < cn[1]; ++iy)
            for (int ix = 0; ix < cn[0]; ++ix) {
              const int c[3] = {cl[0][ix], cl[1][iy], cl[2][iz]};
              if (own_cell(c)) {
                P->sum.push_back(local_e(c, g));
              } else {
                const int64_t cid = c[0] + (int64_t)P->ax[0].n * (c[1] + (int64_t)P->ax[1].n * c[2]);
                P->sum.push_back(-1 - slot.at({gid, cid}));
              }
            }
        P->sum_ptr.push_back((int64_t)P->sum.size());
      }
  // stars: the vertices whose node this rank owns
  const int V[3] = {P->ax[0].n + 1, P->ax[1].n + 1, P->ax[2].n + 1};
  for (int vz = P->cb[4]; vz <= P->cb[5]; ++vz)
    for (int vy = P->cb[2]; vy <= P->cb[3]; ++vy)
      for (int vx = P->cb[0]; vx <= P->cb[1]; ++vx) {
        const int v[3] = {vx, vy, vz};
        bool own = true;
        for (int a = 0; a < 3; ++a) own = own && P->ax[a].rank_of_cell(std::min(v[a], P->ax[a].n - 1)) == P->rc[a];
        if (own) P->stars.push_back(vx + (int64_t)V[0] * (vy + (int64_t)V[1] * vz));
      }
}

}  // namespace

extern "C" {

int fdm_partition_create(int nx, int ny, int nz, int p, int px, int py, int pz, int rank, fdm_partition **out) {
  if (!out) return FDM_EINVAL;
  *out = nullptr;
  if (p < 1 || p > 15 || nx < 1 || ny < 1 || nz < 1 || px < 1 || py < 1 || pz < 1 || px > nx || py > ny || pz > nz ||
      rank < 0 || rank >= px * py * pz) {
    g_part_err = "fdm_partition_create: need 1 <= p <= 15, 1 <= ranks per axis <= cells per axis, 0 <= rank < ranks";
    return FDM_EINVAL;
  }
  fdm_partition *P = new fdm_partition();
  P->p = p;
  P->n = p + 1;
  P->ax[0] = {nx, px};
  P->ax[1] = {ny, py};
  P->ax[2] = {nz, pz};
  P->rank = rank;
  P->rc[0] = rank % px;
  P->rc[1] = (rank / px) % py;
  P->rc[2] = rank / (px * py);
  try {
    build(P);
  } catch (const std::exception &e) {
    g_part_err = std::string("fdm_partition_create: ") + e.what();
    delete P;
    return FDM_ENOMEM;
  }
  *out = P;
  return FDM_OK;
}

int fdm_partition_query(const fdm_partition *P, int what, void *out, size_t *len) {
  if (!P || !out || !len) return FDM_EINVAL;
  auto put = [&](const void *src, size_t bytes) {
    if (*len < bytes) {
      g_part_err = "fdm_partition_query: buffer too small (" + std::to_string(bytes) + " bytes needed)";
      *len = bytes;
      return FDM_EINVAL;
    }
    if (bytes) std::memcpy(out, src, bytes);
    *len = bytes;
    return FDM_OK;
  };
  switch (what) {
    case FDM_PQ_CELL_BOX: return put(P->cb, sizeof P->cb);
    case FDM_PQ_NODE_BOX: return put(P->nb, sizeof P->nb);
    case FDM_PQ_HALO_BOX: return put(P->hb, sizeof P->hb);
    case FDM_PQ_NNEIGH: { int k = (int)P->neigh.size(); return put(&k, sizeof k); }
    case FDM_PQ_NEIGHBORS: return put(P->neigh.data(), P->neigh.size() * sizeof(int));
    case FDM_PQ_SEND_PTR: return put(P->send_ptr.data(), P->send_ptr.size() * sizeof(int64_t));
    case FDM_PQ_SEND: return put(P->send.data(), P->send.size() * sizeof(int64_t));
    case FDM_PQ_RECV_PTR: return put(P->recv_ptr.data(), P->recv_ptr.size() * sizeof(int64_t));
    case FDM_PQ_SUM_PTR: return put(P->sum_ptr.data(), P->sum_ptr.size() * sizeof(int64_t));
    case FDM_PQ_SUM: return put(P->sum.data(), P->sum.size() * sizeof(int64_t));
    case FDM_PQ_OWNED: return put(P->owned.data(), P->owned.size());
    case FDM_PQ_STARS: return put(P->stars.data(), P->stars.size() * sizeof(int64_t));
    default: g_part_err = "fdm_partition_query: unknown quantity"; return FDM_EINVAL;
  }
}

const char *fdm_partition_last_error(void) { return g_part_err.c_str(); }

void fdm_partition_destroy(fdm_partition *P) { delete P; }

}  // extern "C"
