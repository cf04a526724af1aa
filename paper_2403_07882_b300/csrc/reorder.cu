// Reverse Cuthill-McKee locality ordering of the cells on the device (the
// optional internal renumbering; the paper renumbers cells after domain
// decomposition, Sec. 2.3).
//
// Sequence: components in order of their smallest cell; each from a
// George-Liu pseudo-peripheral cell (from the component's smallest cell,
// move to the smallest (degree, index) cell of the last breadth-first level
// while the number of levels grows); Cuthill-McKee appends each visited
// cell's unvisited neighbours by (degree, index); the whole sequence is
// reversed. The FIFO order of Cuthill-McKee is built one level at a time:
// a cell of the next level sits after every cell whose first visited
// neighbour (parent) comes earlier, and among the cells of one parent by
// (degree, index), which is the order the sequential queue produces. Per
// level: discover (parent = smallest position by atomicMin), count per
// parent, scan, place, sort each parent's children, emit. The graph is the
// block-CSR pattern of the structure (rows with their diagonal).
#include <climits>

#include "internal.h"

namespace bcs {
namespace {

__device__ __forceinline__ int degree(const int32_t* __restrict__ rp, int v) { return rp[v + 1] - rp[v] - 1; }

// Cuthill-McKee: the cells of the next level (lvl set to `next` once, by the
// thread that discovers them) and each one's parent position.
__global__ void k_cm_discover(int s0, int m, const int32_t* __restrict__ order, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, int32_t* __restrict__ lvl, int next,
                              int32_t* __restrict__ par, int32_t* __restrict__ nxt, int32_t* __restrict__ nn) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int u = order[s0 + i];
  for (int p = rp[u]; p < rp[u + 1]; ++p) {
    const int v = ci[p];
    if (v == u) continue;
    int old = lvl[v];
    if (old == -1) {
      old = atomicCAS(lvl + v, -1, next);
      if (old == -1) {
        nxt[atomicAdd(nn, 1)] = v;
        old = next;
      }
    }
    if (old == next) atomicMin(par + v, s0 + i);
  }
}

__global__ void k_cm_count(int nn, int s0, const int32_t* __restrict__ nxt, const int32_t* __restrict__ par,
                           int32_t* __restrict__ cnt) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) atomicAdd(cnt + (par[nxt[i]] - s0), 1);
}

__global__ void k_cm_place(int nn, int s0, const int32_t* __restrict__ nxt, const int32_t* __restrict__ par,
                           const int32_t* __restrict__ seg, int32_t* __restrict__ cur, const int32_t* __restrict__ rp,
                           uint64_t* __restrict__ keys) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int v = nxt[i], q = par[v] - s0;
  const int slot = seg[q] + atomicAdd(cur + q, 1);
  keys[slot] = ((uint64_t)(uint32_t)degree(rp, v) << 32) | (uint32_t)v;
}

__global__ void k_cm_emit(int nn, int e0, const uint64_t* __restrict__ keys, int32_t* __restrict__ order) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) order[e0 + i] = (int32_t)(uint32_t)keys[i];
}

// Breadth-first level over cells not yet ordered (lvl == -1); mark holds the
// search's generation. Also the smallest (degree, index) key of the level.
__global__ void k_bfs_step(int m, const int32_t* __restrict__ cur, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const int32_t* __restrict__ lvl, int32_t* __restrict__ mark,
                           int gen, int32_t* __restrict__ nxt, int32_t* __restrict__ nn,
                           unsigned long long* __restrict__ minkey) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int u = cur[i];
  atomicMin(minkey, ((unsigned long long)(uint32_t)degree(rp, u) << 32) | (uint32_t)u);
  for (int p = rp[u]; p < rp[u + 1]; ++p) {
    const int v = ci[p];
    if (v == u || lvl[v] != -1) continue;
    if (atomicExch(mark + v, gen) != gen) nxt[atomicAdd(nn, 1)] = v;
  }
}

__global__ void k_first_unvisited(int C, int from, const int32_t* __restrict__ lvl, int32_t* __restrict__ first) {
  dep_enter();
  const int i = from + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C && lvl[i] == -1) atomicMin(first, i);
}

__global__ void k_reverse(int C, const int32_t* __restrict__ order, int32_t* __restrict__ perm,
                          int32_t* __restrict__ inv) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int old = order[C - 1 - i];
  perm[i] = old;
  inv[old] = i;
}

__global__ void k_start(int r, int pos, int32_t* __restrict__ order, int32_t* __restrict__ lvl, int tag) {
  dep_enter();
  order[pos] = r;
  lvl[r] = tag;
}

}  // namespace

bcs_status rcm_order(Solver* s, const Bsr& A, int32_t* perm, int32_t* inv) {
  const int C = A.rows;
  DBuf<int32_t> lvl, mark, order, par, nxt, cur, cnt, seg, sc;
  DBuf<uint64_t> keys;
  DBuf<unsigned long long> mk;
  BCS_ALLOC(s, lvl, C);
  BCS_ALLOC(s, mark, C);
  BCS_ALLOC(s, order, C);
  BCS_ALLOC(s, par, C);
  BCS_ALLOC(s, nxt, C);
  BCS_ALLOC(s, cur, C);
  BCS_ALLOC(s, cnt, C);
  BCS_ALLOC(s, seg, C + 1);
  BCS_ALLOC(s, keys, C);
  BCS_ALLOC(s, sc, 4);
  BCS_ALLOC(s, mk, 1);
  BCS_CU(s, cudaMemsetAsync(lvl.p, 0xff, C * sizeof(int32_t), s->stream));
  BCS_CU(s, cudaMemsetAsync(mark.p, 0, C * sizeof(int32_t), s->stream));
  BCS_CU(s, cudaMemsetAsync(par.p, 0x7f, C * sizeof(int32_t), s->stream));  // large positive
  const int maxdeg = A.maxrow > 0 ? A.maxrow : 1;
  int placed = 0, from = 0, gen = 0, tag = 0;
  struct Hv {
    int32_t nn;
    int32_t pad;
    unsigned long long minkey;
  };
  // one breadth-first search from r over unordered cells: number of levels
  // and the last level's smallest (degree, index) cell
  auto bfs = [&](int r, int* nlev, int* x) -> bcs_status {
    ++gen;
    const int32_t one = gen;
    BCS_CU(s, cudaMemcpyAsync(mark.p + r, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    BCS_CU(s, cudaMemcpyAsync(cur.p, &r, sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    int m = 1;
    *nlev = 0;
    int32_t* a = cur.p;
    int32_t* b = nxt.p;
    for (;;) {
      ++*nlev;
      BCS_CU(s, cudaMemsetAsync(sc.p, 0, sizeof(int32_t), s->stream));
      BCS_CU(s, cudaMemsetAsync(mk.p, 0xff, sizeof(unsigned long long), s->stream));
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_bfs_step, grid_for(m, 256), 256, 0, m, a, A.rp.p, A.ci.p, lvl.p, mark.p, gen, b,
                 sc.p, mk.p);
      Hv h{};
      BCS_CU(s, cudaMemcpyAsync(&h.nn, sc.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
      BCS_CU(s, cudaMemcpyAsync(&h.minkey, mk.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
      BCS_CU(s, cudaStreamSynchronize(s->stream));
      if (h.nn == 0) {
        *x = (int)(uint32_t)h.minkey;
        return BCS_OK;
      }
      std::swap(a, b);
      m = h.nn;
    }
  };
  while (placed < C) {
    // the component's smallest cell
    int32_t first = INT_MAX;
    BCS_CU(s, cudaMemcpyAsync(sc.p + 1, &first, sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_first_unvisited, grid_for(C - from, 256), 256, 0, C, from, lvl.p, sc.p + 1);
    BCS_CU(s, cudaMemcpyAsync(&first, sc.p + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    if (first == INT_MAX) return s->fail(BCS_EINVAL, "reordering lost a cell");
    from = first;
    // pseudo-peripheral start
    int r = first, nr = 0, x = 0;
    BCS_OKR(bfs(r, &nr, &x));
    for (int guard = 0; guard < C; ++guard) {
      int nx = 0, x2 = 0;
      BCS_OKR(bfs(x, &nx, &x2));
      if (nx <= nr) break;
      r = x;
      nr = nx;
      x = x2;
    }
    // Cuthill-McKee from r, one level at a time
    BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_start, 1, 1, 0, r, placed, order.p, lvl.p, ++tag);
    int s0 = placed, m = 1;
    placed += 1;
    for (;;) {
      const int next = ++tag;
      BCS_CU(s, cudaMemsetAsync(sc.p, 0, sizeof(int32_t), s->stream));
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_cm_discover, grid_for(m, 256), 256, 0, s0, m, order.p, A.rp.p, A.ci.p, lvl.p,
                 next, par.p, nxt.p, sc.p);
      int32_t nn = 0;
      BCS_CU(s, cudaMemcpyAsync(&nn, sc.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
      BCS_CU(s, cudaStreamSynchronize(s->stream));
      if (nn == 0) break;
      BCS_CU(s, cudaMemsetAsync(cnt.p, 0, m * sizeof(int32_t), s->stream));
      BCS_CU(s, cudaMemsetAsync(cur.p, 0, m * sizeof(int32_t), s->stream));
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_cm_count, grid_for(nn, 256), 256, 0, nn, s0, nxt.p, par.p, cnt.p);
      BCS_OKR(exclusive_scan(s, cnt.p, seg.p, m));
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_cm_place, grid_for(nn, 256), 256, 0, nn, s0, nxt.p, par.p, seg.p, cur.p,
                 A.rp.p, keys.p);
      BCS_OKR(segmented_sort64(s, seg.p, keys.p, m, maxdeg));
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_cm_emit, grid_for(nn, 256), 256, 0, nn, s0 + m, keys.p, order.p);
      s0 += m;
      m = nn;
      placed += nn;
    }
  }
  BCS_LAUNCH_DEP(s, K_MISC, 0, 0, k_reverse, grid_for(C, 256), 256, 0, C, order.p, perm, inv);
  return BCS_OK;
}

}  // namespace bcs

// ---- applying the ordering ---------------------------------------------------
namespace bcs {
namespace {

__global__ void k_relabel(int F, const int32_t* __restrict__ inv, const int32_t* __restrict__ o,
                          const int32_t* __restrict__ nb, int32_t* __restrict__ o2, int32_t* __restrict__ nb2) {
  dep_enter();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  o2[f] = inv[o[f]];
  nb2[f] = inv[nb[f]];
}

// Diagonal entries of the LDU maps back in the caller's numbering: the
// source code of row i's diagonal names cell perm[i], and pos_diag is
// indexed by the caller's cell.
__global__ void k_user_diag(int C, const int32_t* __restrict__ perm, const int32_t* __restrict__ pd_new,
                            int32_t* __restrict__ pd_user, int32_t* __restrict__ src) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int p = pd_new[i];
  pd_user[perm[i]] = p;
  src[p] = -1 - perm[i];
}

template <bool GATHER>
__global__ void k_permute_vec(size_t total, int n, const int32_t* __restrict__ perm, const double* __restrict__ in,
                              double* __restrict__ out) {
  dep_enter();
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const size_t i = t / n;
  const size_t k = t - i * n;
  const size_t u = (size_t)perm[i] * n + k;
  if (GATHER)
    out[t] = in[u];
  else
    out[u] = in[t];
}

}  // namespace

bcs_status relabel_faces(Solver* s, const int32_t* o, const int32_t* nb, int32_t* o2, int32_t* nb2) {
  if (s->F > 0)
    BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * s->F, 0, k_relabel, grid_for(s->F, 256), 256, 0, s->F, s->inv.p, o, nb, o2, nb2);
  return BCS_OK;
}

bcs_status user_diag_maps(Solver* s) {
  DBuf<int32_t> pd;
  BCS_ALLOC(s, pd, s->C);
  BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * s->C, 0, k_user_diag, grid_for(s->C, 256), 256, 0, s->C, s->perm.p,
             s->pos_diag.p, pd.p, s->src.p);
  s->pos_diag = std::move(pd);
  return BCS_OK;
}

bcs_status to_internal(Solver* s, const double* user, double* internal) {
  const size_t total = (size_t)s->C * s->n;
  BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total, 0, k_permute_vec<true>, grid_for(total, 256), 256, 0, total, s->n,
             s->perm.p, user, internal);
  return BCS_OK;
}

bcs_status to_user(Solver* s, const double* internal, double* user) {
  const size_t total = (size_t)s->C * s->n;
  BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total, 0, k_permute_vec<false>, grid_for(total, 256), 256, 0, total, s->n,
             s->perm.p, internal, user);
  return BCS_OK;
}

}  // namespace bcs
