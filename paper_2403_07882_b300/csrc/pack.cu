// Segregated fields <-> block AoS on the device (Alg. 1 steps 1, 5 and 15).
//
// A coupled system's unknowns come as a list of fields, field k with
// ncomp[k] components per cell (1: scalar field, 3: vector field stored
// [cell][3]); the block unknown order is the fields' order with each field's
// components in turn. Coefficients come as one coupling per (row field,
// column field) pair: LDU arrays of ncomp[a] x ncomp[b] row-major sub-blocks,
// or nothing (a zero coupling). Pure data movement with coalesced loads and
// stores.
#include "internal.h"

namespace bcs {
namespace {

// Per block component r (0 <= r < n): its field and its index in the field.
struct FieldMap {
  int fof[PK_MAX_FIELDS];
  int loc[PK_MAX_FIELDS];
  int nc[PK_MAX_FIELDS];
};

FieldMap field_map(int nfields, const int* ncomp) {
  FieldMap m{};
  int r = 0;
  for (int k = 0; k < nfields; ++k) {
    for (int j = 0; j < ncomp[k]; ++j, ++r) {
      m.fof[r] = k;
      m.loc[r] = j;
    }
    m.nc[k] = ncomp[k];
  }
  return m;
}

struct VecTable {
  const double* in[PK_MAX_FIELDS];
  double* out[PK_MAX_FIELDS];
};

template <int N, bool PACK>
__global__ void k_pack_vector(size_t total, FieldMap m, VecTable t, const double* __restrict__ vin,
                              double* __restrict__ vout) {
  dep_enter();
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t c = i / N;
  const int r = (int)(i - c * N);
  const int k = m.fof[r];
  const size_t j = c * m.nc[k] + m.loc[r];
  if (PACK)
    vout[i] = __ldg(t.in[k] + j);
  else
    t.out[k][j] = __ldg(vin + i);
}

struct CoefTable {
  const double* src[PK_MAX_FIELDS * PK_MAX_FIELDS][3];  // [a * nf + b][diag, upper, lower]
  int nf;
};

// Coefficients: one warp per tile of pk_tile<N> consecutive blocks of one kind
// (diag, upper or lower). The warp copies each coupling's sub-blocks of the
// tile (contiguous in the coupling's array) into the tile's place in shared
// memory, then writes the tile out: contiguous in the LDU arrays, one n x n
// block at a time into the solver's block-CSR values. Zero couplings stay
// zero. Reads and writes are coalesced.
constexpr int PK_WARPS = 4;
constexpr int PK_U = 4;
template <int N>
constexpr int pk_tile() {
  return N >= 7 ? 16 : 32;  // static shared memory of a block <= 48 KB
}

template <int N, bool BSR>
__global__ void __launch_bounds__(PK_WARPS * 32) k_pack_coefficients(int C, int F, FieldMap m, CoefTable t,
                                                                     const int32_t* __restrict__ pos_diag,
                                                                     const int32_t* __restrict__ pos_up,
                                                                     const int32_t* __restrict__ pos_lo,
                                                                     double* __restrict__ diag,
                                                                     double* __restrict__ upper,
                                                                     double* __restrict__ lower,
                                                                     double* __restrict__ val) {
  dep_enter();
  constexpr int NN = N * N, PK_TILE = pk_tile<N>();
  __shared__ double tile_s[PK_WARPS][PK_TILE * NN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* tile = tile_s[warp];
  const long long w = (long long)blockIdx.x * PK_WARPS + warp;
  const long long td = (C + PK_TILE - 1) / PK_TILE, tf = (F + PK_TILE - 1) / PK_TILE;
  int kind, cnt;
  long long i0;
  if (w < td) {
    kind = 0;
    i0 = w * PK_TILE;
    cnt = (int)min((long long)PK_TILE, (long long)C - i0);
  } else if (w < td + tf) {
    kind = 1;
    i0 = (w - td) * PK_TILE;
    cnt = (int)min((long long)PK_TILE, (long long)F - i0);
  } else if (w < td + 2 * tf) {
    kind = 2;
    i0 = (w - td - tf) * PK_TILE;
    cnt = (int)min((long long)PK_TILE, (long long)F - i0);
  } else {
    return;
  }
  for (int i = lane; i < cnt * NN; i += 32) tile[i] = 0.0;
  __syncwarp();
  int r0 = 0;
  for (int a = 0; a < t.nf; ++a) {
    const int na = m.nc[a];
    int c0 = 0;
    for (int b = 0; b < t.nf; ++b) {
      const int nb = m.nc[b], sz = na * nb;
      const double* src = t.src[a * t.nf + b][kind];
      if (src) {
        // PK_U loads in flight per lane, then their places in the tile
        const double* base = src + i0 * sz;
        const int tot = cnt * sz;
        for (int i = lane; i < tot; i += 32 * PK_U) {
          double v[PK_U];
#pragma unroll
          for (int u = 0; u < PK_U; ++u) v[u] = i + 32 * u < tot ? __ldg(base + i + 32 * u) : 0.0;
#pragma unroll
          for (int u = 0; u < PK_U; ++u) {
            const int j = i + 32 * u;
            if (j >= tot) break;
            const int bl = j / sz, rem = j - bl * sz, ra = rem / nb, cb = rem - ra * nb;
            tile[bl * NN + (r0 + ra) * N + c0 + cb] = v[u];
          }
        }
      }
      c0 += nb;
    }
    r0 += na;
  }
  __syncwarp();
  if (BSR) {
    const int32_t* pos = kind == 0 ? pos_diag : (kind == 1 ? pos_up : pos_lo);
    for (int i = lane; i < cnt * NN; i += 32) {
      const int bl = i / NN, e = i - bl * NN;
      val[(size_t)__ldg(pos + i0 + bl) * NN + e] = tile[i];
    }
  } else {
    double* o = (kind == 0 ? diag : (kind == 1 ? upper : lower)) + i0 * NN;
    for (int i = lane; i < cnt * NN; i += 32) o[i] = tile[i];
  }
}

}  // namespace

bcs_status pack_vector(Solver* s, int nfields, const int* ncomp, const double* const* fields, double* out) {
  const FieldMap m = field_map(nfields, ncomp);
  VecTable t{};
  for (int k = 0; k < nfields; ++k) t.in[k] = fields[k];
  const size_t total = (size_t)s->C * s->n;
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total, 0, (k_pack_vector<N, true>), grid_for(total, 256), 256, 0, total, m, t,
               (const double*)nullptr, out);
    return BCS_OK;
  });
}

bcs_status unpack_vector(Solver* s, int nfields, const int* ncomp, const double* in, double* const* fields) {
  const FieldMap m = field_map(nfields, ncomp);
  VecTable t{};
  for (int k = 0; k < nfields; ++k) t.out[k] = fields[k];
  const size_t total = (size_t)s->C * s->n;
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total, 0, (k_pack_vector<N, false>), grid_for(total, 256), 256, 0, total, m,
               t, in, (double*)nullptr);
    return BCS_OK;
  });
}

bcs_status pack_coefficients(Solver* s, int nfields, const int* ncomp, const double* const* src, double* diag,
                             double* upper, double* lower) {
  const FieldMap m = field_map(nfields, ncomp);
  CoefTable t{};
  t.nf = nfields;
  for (int p = 0; p < nfields * nfields; ++p)
    for (int k = 0; k < 3; ++k) t.src[p][k] = src[3 * p + k];
  const int C = s->C, F = s->F, n = s->n;
  const bool bsr = !diag;
  if (bsr) BCS_ALLOC(s, s->lv[0].A.v, (size_t)s->lv[0].A.nnz * n * n);
  double* val = bsr ? s->lv[0].A.v.p : nullptr;
  const size_t total = ((size_t)C + 2 * (size_t)F) * n * n;
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value, T = pk_tile<N>();
    const size_t tiles = ((size_t)C + T - 1) / T + 2 * (((size_t)F + T - 1) / T);
    const unsigned grid = grid_for(tiles, PK_WARPS);
    if (bsr)
      BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total + 4.0 * (C + 2.0 * F), 0, (k_pack_coefficients<N, true>), grid,
                 PK_WARPS * 32, 0, C, F, m, t, s->pos_diag.p, s->pos_up.p, s->pos_lo.p, nullptr, nullptr, nullptr,
                 val);
    else
      BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * total, 0, (k_pack_coefficients<N, false>), grid, PK_WARPS * 32, 0, C, F, m,
                 t, nullptr, nullptr, nullptr, diag, upper, lower, nullptr);
    return BCS_OK;
  });
}

}  // namespace bcs
