// FP64 CPU oracle: reverse Cuthill-McKee locality ordering of the cells
// (the internal renumbering that stands in for Sec. 2.3's renumbering after
// decomposition).
//
// TEST INFRASTRUCTURE ONLY (see oracle.h). Textbook sequential algorithm:
//   * the cell graph has an edge per face;
//   * components are taken in order of their smallest cell index;
//   * each component starts from a pseudo-peripheral cell (George and Liu):
//     from the component's smallest index r, a breadth-first search; x = the
//     cell of the last level with the smallest (degree, index); if x's search
//     has more levels than r's, r = x and repeat;
//   * Cuthill-McKee: a FIFO queue from r; each dequeued cell appends its
//     unvisited neighbours by (degree, index) ascending;
//   * the whole sequence reversed: perm[new] = old.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "oracle.h"

namespace {

struct Graph {
  std::vector<std::vector<int>> adj;
  int deg(int v) const { return (int)adj[v].size(); }
};

// levels of a breadth-first search from r over unvisited cells; returns the
// number of levels and the last level's cells
int bfs_levels(const Graph& g, const std::vector<char>& done, int r, std::vector<int>& last) {
  std::vector<int> level(g.adj.size(), -1);
  std::vector<int> cur{r}, next;
  level[r] = 0;
  int nlev = 0;
  while (!cur.empty()) {
    ++nlev;
    last = cur;
    next.clear();
    for (int u : cur)
      for (int v : g.adj[u])
        if (!done[v] && level[v] < 0) {
          level[v] = nlev;
          next.push_back(v);
        }
    cur.swap(next);
  }
  return nlev;
}

int smallest_by_degree(const Graph& g, const std::vector<int>& cells) {
  int best = cells[0];
  for (int v : cells)
    if (g.deg(v) < g.deg(best) || (g.deg(v) == g.deg(best) && v < best)) best = v;
  return best;
}

}  // namespace

extern "C" int or_rcm(int C, int F, const int32_t* owner, const int32_t* nb, int32_t* perm) {
  Graph g;
  g.adj.assign(C, {});
  for (int f = 0; f < F; ++f) {
    if (owner[f] < 0 || owner[f] >= C || nb[f] < 0 || nb[f] >= C || owner[f] == nb[f]) return 1;
    g.adj[owner[f]].push_back(nb[f]);
    g.adj[nb[f]].push_back(owner[f]);
  }
  for (auto& a : g.adj) std::sort(a.begin(), a.end());
  std::vector<char> done(C, 0);
  std::vector<int> order;
  order.reserve(C);
  for (int s = 0; s < C; ++s) {
    if (done[s]) continue;
    // pseudo-peripheral start
    int r = s;
    std::vector<int> last;
    int nr = bfs_levels(g, done, r, last);
    for (;;) {
      const int x = smallest_by_degree(g, last);
      std::vector<int> lx;
      const int nx = bfs_levels(g, done, x, lx);
      if (nx <= nr) break;
      r = x;
      nr = nx;
      last = lx;
    }
    // Cuthill-McKee from r
    size_t head = order.size();
    order.push_back(r);
    done[r] = 1;
    while (head < order.size()) {
      const int u = order[head++];
      std::vector<int> nbrs;
      for (int v : g.adj[u])
        if (!done[v]) nbrs.push_back(v);
      std::sort(nbrs.begin(), nbrs.end(), [&](int a, int b) {
        return g.deg(a) != g.deg(b) ? g.deg(a) < g.deg(b) : a < b;
      });
      for (int v : nbrs) {
        done[v] = 1;
        order.push_back(v);
      }
    }
  }
  for (int i = 0; i < C; ++i) perm[i] = order[C - 1 - i];
  return 0;
}
