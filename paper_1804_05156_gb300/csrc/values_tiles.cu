// Two-phase value path in float-float arithmetic: every element is computed exactly once, and every
// row sums its incidences in ascending element order.
//
// Phase 1 (k_tile_elements): one CTA per tile of TE elements in locality order (tileplan.cu). The
//   tile's vertices are staged in shared memory once (exact three-float splits; for the 2-D
//   sine-product load also sin/cos(pi x/2) per coordinate), then each thread computes one element's
//   local stiffness and load entries (element_df.cuh: Sec. 3.1.3, eq. (dlambda), Sec. 3.2) and writes,
//   for each local row i, one packet of float pairs to the slot q of incidence (t, i):
//     2-D: (a_ij, a_ik) 16 bytes at pair array [q] and b_i 8 bytes at load array [q] (24 bytes, both
//          stores aligned: no divergent paths); in the fused form, where the gather reads the packets
//          back through L2 in the same launch, (a_ij, a_ik, b_i, unused) as 32 bytes in one 256-bit store;
//     3-D: (a_ij, a_ik, a_il, b_i), 32 bytes in one 256-bit store,
//   with j < k < l the other local indices. The diagonal is re-formed from the packet in phase 2 exactly
//   as the element routine forms it (2-D a_ii = -(a_ij + a_ik), 3-D ((0 - a_ij) - a_ik) - a_il), so it
//   costs no bytes.
// Phase 2 (k_row_gather): one thread per row, one warp per 32 consecutive rows. A row's packets are
//   contiguous (the incidence lists are sorted by row, then element). Each thread adds its row's
//   diagonal and load terms in registers and the off-diagonal terms in the warp's shared-memory copy
//   of its 32 rows (CSR order); the warp then converts and writes the rows with coalesced stores.
// Fused form (k_tiles_fused): both phases in one cooperative launch of resident CTAs. Tiles, then
//   groups of rows, are taken from device counters; between the phases a grid-wide barrier (an
//   arrival counter, polled with a bounded wait) orders every packet write before any read.
// Every CSR entry is the float-float sum of its element contributions in ascending element order,
// rounded to double once, whatever the tile size or launch form: the same bits as the owner-computes
// kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "element_df.cuh"
#include "packet.cuh"

namespace fem {

const float4* sincos_table_device();  // values_blocked.cu

namespace {

struct TileArgs {
  int64_t NT;
  int ntiles;
  const int32_t* elist;
  const uint16_t* lelem;
  const int32_t* voff;
  const int32_t* vlist;
  const int32_t* ipos;
  float4* pk;
  int xs_bytes;
  int op;               // kOpStiffness (with the load vector), kOpMass or kOpAniso (values only), kOpApply
  const double* opk;    // operator coefficients: mass c [NT] (nullable), aniso tensor [NT][d(d+1)/2]
  const double* u;      // kOpApply: the vector A is applied to [N]
  const uint8_t* isbd;  // kOpApply: eliminated (Dirichlet) vertices, nullable
  int u_off;            // kOpApply: shared-memory offset of the staged u values
  int bar_extra;        // fused form: arrivals the grid barrier waits for beyond the launch's CTAs (0)
  int bar_polls;        // fused form: polls before the grid barrier gives up
};

struct RowArgs {
  int64_t N;
  int max_row;
  const int32_t* row_ptr;
  const int32_t* inc_ptr;
  const void* pw;
  const uint8_t* rdp;
  const float4* pk;
  const float2* pkb;    // 2-D: the load (or mass-diagonal) terms, one pair per incidence
  bool diag_in_packet;  // the packet's last pair is the diagonal entry (mass matrix), not a load term
};

// Staged 2-D record: the coordinates and, for the sine-product load, the vertex's sine products
// (sin_products), 48 bytes (three 16-byte bank groups): a warp's scattered reads of the records of
// different vertices fall on all eight 16-byte groups of banks instead of four.
struct __align__(16) Vtx2 {
  VtxDF<2> v;
  df2 P[4];
};
template <int D>
__host__ __device__ constexpr int staged_vtx_bytes() { return D == 2 ? (int)sizeof(Vtx2) : (int)sizeof(VtxDF<3>); }

// Phase 1 for one tile (all TE threads of the CTA; one __syncthreads inside).
template <int D, int TE, bool FUSED = false>
__device__ __forceinline__ void elements_of_tile(const TileArgs& a, int tile, unsigned char* sm,
                                                 const double* __restrict__ node, const double* __restrict__ k,
                                                 int f_kind, const double* __restrict__ f_arg, int want_a, int want_b,
                                                 const float4* __restrict__ tab, int* __restrict__ err) {
  constexpr int D1 = D + 1;
  VtxDF<D>* xs = reinterpret_cast<VtxDF<D>*>(sm);  // 3-D; 2-D stages VtxPad2 / SCPad2 records
  const int v0 = __ldg(a.voff + tile), nv = __ldg(a.voff + tile + 1) - v0;
  const bool sinprod2 = (D == 2) && f_kind == FEM_F_SINPROD && want_b;
  // element data first: its loads are in flight during the vertex staging
  const int64_t j = (int64_t)tile * TE + threadIdx.x;
  const bool act = j < a.NT;
  int t = 0;
  int lv[D1], qi[D1];
  double kd = 1.0;
  if (act) {
    t = __ldg(a.elist + j);
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      lv[i] = __ldg(a.lelem + (int64_t)i * a.NT + j);
      qi[i] = __ldg(a.ipos + (int64_t)i * a.NT + j);
    }
    if (k && want_a) kd = __ldg(k + t);
  }
  for (int v = threadIdx.x; v < nv; v += TE) {
    const int R = __ldg(a.vlist + v0 + v);
    VtxDF<D> x;
    stage_vertex<D>(x, node + (size_t)R * D);
    if constexpr (D == 2) {
      Vtx2* rec = reinterpret_cast<Vtx2*>(sm) + v;
      rec->v = x;
      if (sinprod2) sin_products(sincospi_half(split3(x.x[0]), tab), sincospi_half(split3(x.x[1]), tab), rec->P);
    } else {
      xs[v] = x;
    }
    if (a.op == kOpApply)  // eliminated vertices contribute nothing to the free rows
      reinterpret_cast<df2*>(sm + a.u_off)[v] =
          (a.isbd && __ldg(a.isbd + R)) ? df2{0.0f, 0.0f} : df_from_double(__ldg(a.u + R));
  }
  __syncthreads();
  if (!act) return;
  int st = FEM_OK;
  const df2 kt = (k && want_a) ? coef_df(kd, st) : df2{1.0f, 0.0f};
  const df2 fconst = (f_kind == FEM_F_CONST && f_arg) ? coef_df(__ldg(f_arg), st) : df2{1.0f, 0.0f};
  LocalDF<D> L;
#pragma unroll
  for (int c = 0; c < D1 * (D1 + 1) / 2; ++c) L.a[c] = df2{0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < D1; ++i) L.bt[i] = df2{0.0f, 0.0f};
  const VtxDF<D>* V[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) {
    if constexpr (D == 2) V[i] = &(reinterpret_cast<const Vtx2*>(sm) + lv[i])->v;
    else V[i] = &xs[lv[i]];
  }
  if (a.op == kOpMass || a.op == kOpAniso) {
    const double* c = (a.op == kOpMass) ? (a.opk ? a.opk + t : nullptr) : a.opk + (size_t)t * (D * D1 / 2);
    st = worst(st, element_df_operator<D>(reinterpret_cast<const VtxDF<D>* const(&)[D1]>(V), a.op, c, L));
    if (a.op == kOpMass) {
#pragma unroll
      for (int i = 0; i < D1; ++i) L.bt[i] = L.a[i];  // the diagonal travels in the load slot
    }
  } else if constexpr (D == 2) {
    const Vtx2* rec = reinterpret_cast<const Vtx2*>(sm);
    const VtxDF<2>* const V2[3] = {V[0], V[1], V[2]};
    const df2* const Pv[3] = {rec[lv[0]].P, rec[lv[1]].P, rec[lv[2]].P};
    st = worst(st, element_df2(V2, Pv, kt, want_a, want_b, f_kind, fconst, f_arg, t, L, false));  // diagonals: in the gather
  } else {
    const VtxDF<3>* const V3[4] = {V[0], V[1], V[2], V[3]};
    st = worst(st, element_df3(V3, kt, want_a, want_b, f_kind, fconst, f_arg, t, tab, L, false));  // diagonals: in the gather
  }
  if (st != FEM_OK) report(err, st);
  if (a.op == kOpApply) {
    // (A u)_i contribution of the element: sum_{j != i} a_ij (u_j - u_i), since a_ii = -sum_{j != i} a_ij
    const df2* ux = reinterpret_cast<const df2*>(sm + a.u_off);
    df2 uu[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) uu[i] = ux[lv[i]];
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      df2 y = {0.0f, 0.0f};
#pragma unroll
      for (int jj = 0; jj < D1; ++jj)
        if (jj != i) y = df_add(y, df_mul(L.a[pidx<D>(i, jj)], df_sub(uu[jj], uu[i])));
      reinterpret_cast<float2*>(a.pk)[qi[i]] = make_float2(y.h, y.l);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < D1; ++i) {
    df2 o[D];  // a_ij for the other local indices j, ascending
    int c = 0;
#pragma unroll
    for (int jj = 0; jj < D1; ++jj)
      if (jj != i) o[c++] = L.a[pidx<D>(i, jj)];
    if constexpr (D == 2) {
      // 2-D packet in two arrays: (a_ij, a_ik) 16 bytes at pk[q], b_i 8 bytes at the load array's [q]
      if constexpr (FUSED) {  // read back through L2 in the same launch: one 256-bit access per packet
        store_packet32(a.pk + 2 * (size_t)qi[i], make_float4(o[0].h, o[0].l, o[1].h, o[1].l),
                       make_float4(L.bt[i].h, L.bt[i].l, 0.0f, 0.0f));
      } else {  // a stiffness-only or load-only call writes (and its gather reads) only its own array
        if (want_a) a.pk[qi[i]] = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
        if (want_b || a.op == kOpMass)  // the mass matrix's diagonal travels in the load slot
          reinterpret_cast<float2*>(a.pk + a.NT * 3)[qi[i]] = make_float2(L.bt[i].h, L.bt[i].l);
      }
    } else {
      store_packet32(a.pk + 2 * (size_t)qi[i], make_float4(o[0].h, o[0].l, o[1].h, o[1].l),
                     make_float4(o[2].h, o[2].l, L.bt[i].h, L.bt[i].l));
    }
  }
}

// One packet into a row's sums: the diagonal and load terms in registers, the off-diagonal terms in the
// warp's shared-memory copy of its rows. w holds the in-row positions of the other columns, 8 bits each.
template <int D>
__device__ __forceinline__ void add_packet(const float4& p0, const float4& p1, uint32_t w, int o, df2* acc, df2& dacc,
                                           df2& bacc, bool want_a, bool want_b, bool diag_in_packet = false) {
  if (want_a) {
    const int c0 = o + (int)(w & 0xffu), c1 = o + (int)((w >> 8) & 0xffu);
    if constexpr (D == 2) {
      const df2 o1 = {p0.x, p0.y}, o2 = {p0.z, p0.w};
      // a_ii = -(a_ij + a_ik), as the element routine forms it (or carried in the packet)
      dacc = df_acc(dacc, diag_in_packet ? df2{p1.x, p1.y} : df_neg(df_add(o1, o2)));
      acc[c0] = df_acc(acc[c0], o1);
      acc[c1] = df_acc(acc[c1], o2);
    } else {
      const df2 o1 = {p0.x, p0.y}, o2 = {p0.z, p0.w}, o3 = {p1.x, p1.y};
      const int c2 = o + (int)((w >> 16) & 0xffu);
      dacc = df_acc(dacc, diag_in_packet ? df2{p1.z, p1.w} : df_sub(df_sub(df_sub(df2{0.0f, 0.0f}, o1), o2), o3));
      acc[c0] = df_acc(acc[c0], o1);
      acc[c1] = df_acc(acc[c1], o2);
      acc[c2] = df_acc(acc[c2], o3);
    }
  }
  if (want_b) {
    if constexpr (D == 2) bacc = df_acc(bacc, df2{p1.x, p1.y});
    else bacc = df_acc(bacc, df2{p1.z, p1.w});
  }
}

// packet load: read-only path in the two-launch form; L2 (coherent) path when the packets were written
// earlier in the same launch
template <bool FRESH>
__device__ __forceinline__ float4 load_packet_half(const float4* p) {
  if constexpr (FRESH) return __ldcg(p);
  else return __ldg(p);
}
template <bool FRESH>
__device__ __forceinline__ float2 load_pair(const float2* p) {
  if constexpr (FRESH) return __ldcg(p);
  else return __ldg(p);
}
// packet q as (p0, p1): 2-D (a_ij, a_ik) and b_i from their two arrays, 3-D four pairs (32 bytes)
template <int D, bool FRESH>
__device__ __forceinline__ void load_packet(const float4* pk, const float2* pkb, int64_t q, float4& p0, float4& p1,
                                            bool want_a, bool want_b) {
  if constexpr (D == 2 && FRESH) {
    // fused form: 32-byte packets (a_ij, a_ik, b_i, unused) in one 256-bit load
    load_packet32<FRESH>(pk + 2 * q, p0, p1);
  } else if constexpr (D == 2) {
    // two-launch form: (a_ij, a_ik) from the pair array, b_i from the load array: two aligned loads. A
    // stiffness-only or load-only call writes only its own array; the other load then reads entry 0 over
    // and over (an L1 hit; add_packet ignores the value)
    p0 = load_packet_half<FRESH>(pk + (want_a ? q : 0));
    const float2 z = load_pair<FRESH>(pkb + (want_b ? q : 0));
    p1 = make_float4(z.x, z.y, 0.0f, 0.0f);
  } else {
    load_packet32<FRESH>(pk + 2 * q, p0, p1);
  }
}

// Phase 2 for the 32 rows R0 .. R0+31 of one warp. A row's packets are contiguous; each thread loads U
// of them before adding them in order, so several loads are in flight per thread.
template <int D, typename PW, bool FRESH>
__device__ __forceinline__ void rows_of_warp(const RowArgs& g, int64_t R0, df2* acc, double* __restrict__ val,
                                             double* __restrict__ bvec) {
  constexpr int U = 3;  // measured: 2-D 3 against 2 and 4, 3-D 3 against 2, 4 and 6
  const PW* __restrict__ pw = static_cast<const PW*>(g.pw);
  const int lane = threadIdx.x & 31;
  const int64_t R = R0 + lane;
  const bool act = R < g.N;
  const int64_t Rend = (R0 + 32 < g.N) ? R0 + 32 : g.N;
  const int base = __ldg(g.row_ptr + R0);
  const int region = __ldg(g.row_ptr + Rend) - base;
  const bool want_a = val != nullptr, want_b = bvec != nullptr;
  if (want_a)
    for (int x = lane; x < region; x += 32) acc[x] = df2{0.0f, 0.0f};
  __syncwarp();
  if (act) {
    const int rp = __ldg(g.row_ptr + R), rl = __ldg(g.row_ptr + R + 1) - rp;
    const int o = rp - base;
    df2 dacc = {0.0f, 0.0f}, bacc = {0.0f, 0.0f};
    const int q1 = __ldg(g.inc_ptr + R + 1);
    int q = __ldg(g.inc_ptr + R);
    for (; q + U - 1 < q1; q += U) {
      float4 x0[U], x1[U];
      uint32_t w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        load_packet<D, FRESH>(g.pk, g.pkb, q + u, x0[u], x1[u], want_a, want_b || g.diag_in_packet);
        w[u] = (uint32_t)__ldg(pw + q + u);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) add_packet<D>(x0[u], x1[u], w[u], o, acc, dacc, bacc, want_a, want_b, g.diag_in_packet);
    }
    for (; q < q1; ++q) {
      float4 x0, x1;
      load_packet<D, FRESH>(g.pk, g.pkb, q, x0, x1, want_a, want_b || g.diag_in_packet);
      add_packet<D>(x0, x1, (uint32_t)__ldg(pw + q), o, acc, dacc, bacc, want_a, want_b, g.diag_in_packet);
    }
    if (want_a && rl > 0) acc[o + __ldg(g.rdp + R)] = dacc;
    if (want_b) bvec[R] = df_to_double(bacc);
  }
  __syncwarp();
  if (want_a)
    for (int x = lane; x < region; x += 32) val[base + x] = df_to_double(acc[x]);
  __syncwarp();
}

// Registers capped so that CTAS 128-thread tiles fit an SM: ten in 2-D (no spills), seven in 3-D (a few
// spilled bytes cost less than the lost occupancy); the 3-D sine-product load, whose twelve sine
// evaluations hold more registers, runs six (measured on the 64^3 mesh: 0.174 against 0.185 ms for
// seven and 0.195 for eight; with f = 1 seven stay best, 0.680 against 0.692 ms for six on 128^3).
template <int D, int TE, int CTAS = (D == 3 ? 7 : 10)>
__global__ void __launch_bounds__(TE, CTAS * 128 / TE)
    k_tile_elements(TileArgs a, const double* __restrict__ node, const double* __restrict__ k, int f_kind,
                    const double* __restrict__ f_arg, int want_a, int want_b, const float4* __restrict__ tab,
                    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sm[];
  elements_of_tile<D, TE>(a, blockIdx.x, sm, node, k, f_kind, f_arg, want_a, want_b, tab, err);
}

template <int D, typename PW>
__global__ void __launch_bounds__(256) k_row_gather(RowArgs g, double* __restrict__ val, double* __restrict__ bvec) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int wid = threadIdx.x >> 5;
  const int64_t R0 = (int64_t)blockIdx.x * blockDim.x + wid * 32;
  if (R0 >= g.N) return;  // whole warp
  rows_of_warp<D, PW, false>(g, R0, reinterpret_cast<df2*>(sm) + (size_t)wid * 32 * g.max_row, val, bvec);
}

// y = A u: per row, its element contributions in ascending element order; eliminated rows give u
__global__ void __launch_bounds__(256) k_apply_gather(int64_t N, const int32_t* __restrict__ inc_ptr,
                                                      const float2* __restrict__ pk, const double* __restrict__ u,
                                                      const uint8_t* __restrict__ isbd, double* __restrict__ y) {
  const int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= N) return;
  if (isbd && __ldg(isbd + R)) {
    y[R] = __ldg(u + R);
    return;
  }
  df2 acc = {0.0f, 0.0f};
  const int q1 = __ldg(inc_ptr + R + 1);
  int q = __ldg(inc_ptr + R);
  for (; q + 1 < q1; q += 2) {
    const float2 a = __ldg(pk + q), b = __ldg(pk + q + 1);
    acc = df_acc(acc, df2{a.x, a.y});
    acc = df_acc(acc, df2{b.x, b.y});
  }
  if (q < q1) {
    const float2 a = __ldg(pk + q);
    acc = df_acc(acc, df2{a.x, a.y});
  }
  y[R] = df_to_double(acc);
}

constexpr int kBarrierPolls = 1 << 24;  // bounded grid-barrier wait (with a short sleep per poll)
constexpr int kItemsPerClaim = 8;       // tiles (or row groups) taken per counter increment

// ctr[0]: next tile, ctr[1]: CTAs past phase 1, ctr[2]: next group of TE rows (taken kItemsPerClaim at a
// time); zeroed before the launch. 2-D: registers capped so that ten 128-thread CTAs are resident per
// SM, as for the element kernel; 3-D six.
template <int D, int TE, typename PW>
__global__ void __launch_bounds__(TE, (D == 3 ? 768 : 1280) / TE)
    k_tiles_fused(TileArgs a, RowArgs g, const double* __restrict__ node, const double* __restrict__ k, int f_kind,
                  const double* __restrict__ f_arg, double* __restrict__ val, double* __restrict__ bvec,
                  const float4* __restrict__ tab, int* __restrict__ ctr, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_item;
  const int want_a = val != nullptr, want_b = bvec != nullptr;
  for (;;) {
    __syncthreads();  // the previous tiles are done with the staged vertices and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr[0], kItemsPerClaim);
    __syncthreads();
    const int first = s_item;
    if (first >= a.ntiles) break;
    const int last = min(first + kItemsPerClaim, a.ntiles);
    for (int tile = first; tile < last; ++tile) {
      if (tile > first) __syncthreads();  // staging of the next tile overwrites shared memory
      elements_of_tile<D, TE, true>(a, tile, sm, node, k, f_kind, f_arg, want_a, want_b, tab, err);
    }
  }
  // grid-wide barrier: every packet of every tile is written before any row reads one
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&ctr[1], 1);
    int polls = 0;
    const int target = (int)gridDim.x + a.bar_extra;
    while (*(volatile int*)&ctr[1] < target && polls < a.bar_polls) {
      __nanosleep(64);
      ++polls;
    }
    __threadfence();
    s_item = (polls < a.bar_polls) ? 0 : -1;
  }
  __syncthreads();
  if (s_item < 0) {
    if (threadIdx.x == 0) report(err, FEM_ERR_TIMEOUT);
    return;
  }
  const int wid = threadIdx.x >> 5;
  df2* acc = reinterpret_cast<df2*>(sm) + (size_t)wid * 32 * g.max_row;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(&ctr[2], kItemsPerClaim);
    __syncthreads();
    const int64_t G0 = (int64_t)s_item * TE;
    if (G0 >= g.N) break;
    for (int c = 0; c < kItemsPerClaim; ++c) {
      const int64_t R0 = G0 + (int64_t)c * TE + wid * 32;
      if (R0 < g.N) rows_of_warp<D, PW, true>(g, R0, acc, val, bvec);
    }
  }
}

__host__ __device__ constexpr int gather_warp_bytes(int max_row) { return 32 * max_row * (int)sizeof(df2); }

// warps per CTA of the gather: as many (up to 8) as fit 48 KB of row copies
int gather_warps(int max_row) {
  const int w = (48 * 1024) / gather_warp_bytes(max_row > 0 ? max_row : 1);
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

}  // namespace

int tile_smem_need(const TilePlan& T, int d, bool) {
  return ((T.max_v * (d == 2 ? staged_vtx_bytes<2>() : staged_vtx_bytes<3>())) + 15) / 16 * 16;
}

// Shared memory of the fused kernel (staging of phase 1 or row copies of phase 2, whichever is larger);
// 0 if it exceeds what one CTA may use.
int tile_fused_smem(const TilePlan& T, int d) {
  const int mr = T.max_row > 0 ? T.max_row : 1;
  const int need = std::max(tile_smem_need(T, d, true), (T.TE / 32) * gather_warp_bytes(mr));
  return need <= 200 * 1024 ? need : 0;
}

int assemble_tiles(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg, double* val,
                   double* b, cudaStream_t s, int op, const double* opk, const double* u, const uint8_t* isbd,
                   double* y) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  const float4* tab = sincos_table_device();
  if (!tab) return set_error(FEM_ERR_CUDA, "sin/cos table unavailable");
  const TilePlan& T = P->tile;
  const int D = P->d;
  if (P->NT == 0 || T.ntiles == 0) {
    if (val && P->nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P->nnz, s));
    if (b && P->N > 0) FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * P->N, s));
    return FEM_OK;
  }
  if (reinterpret_cast<uintptr_t>(T.pk) & 31) return set_error(FEM_ERR_STATE, "packet buffer not 32-byte aligned");
  TileArgs a{};
  a.NT = P->NT;
  a.ntiles = T.ntiles;
  a.elist = T.elist;
  a.lelem = T.lelem;
  a.voff = T.voff;
  a.vlist = T.vlist;
  a.ipos = T.ipos;
  a.pk = T.pk;
  a.xs_bytes = ((T.max_v * (D == 2 ? staged_vtx_bytes<2>() : staged_vtx_bytes<3>())) + 15) / 16 * 16;
  a.op = op;
  a.opk = opk;
  a.u = u;
  a.isbd = isbd;
  a.bar_extra = P->bar_extra;
  a.bar_polls = P->bar_polls > 0 ? P->bar_polls : kBarrierPolls;
  if (op != kOpStiffness) {
    b = nullptr;  // operators give values only
    f_kind = FEM_F_CONST;
  }
  RowArgs g;
  g.N = P->N;
  g.max_row = T.max_row > 0 ? T.max_row : 1;
  g.row_ptr = P->row_ptr;
  g.inc_ptr = P->inc_ptr;
  g.pw = T.pw;
  g.rdp = T.rdp;
  g.pk = T.pk;
  g.pkb = reinterpret_cast<const float2*>(T.pk + P->NT * 3);
  g.diag_in_packet = op == kOpMass;
  const int want_a = val != nullptr || op == kOpApply, want_b = b != nullptr;
  if (op == kOpApply) {
    a.u_off = ((tile_smem_need(T, D, false)) + 15) / 16 * 16;
    const int smem = a.u_off + T.max_v * (int)sizeof(df2);
#define FEM_APPLY_LAUNCH(DD, TT)                                                                              \
  do {                                                                                                        \
    if (smem > 48 * 1024)                                                                                     \
      FEM_CUDA(cudaFuncSetAttribute(k_tile_elements<DD, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
    FEM_LAUNCH((k_tile_elements<DD, TT>), T.ntiles, TT, smem, s, a, node, k, FEM_F_CONST, nullptr, 1, 0, tab, err); \
  } while (0)
    if (D == 2) {
      if (T.TE == 128) FEM_APPLY_LAUNCH(2, 128);
      else FEM_APPLY_LAUNCH(2, 256);
    } else {
      if (T.TE == 128) FEM_APPLY_LAUNCH(3, 128);
      else FEM_APPLY_LAUNCH(3, 256);
    }
#undef FEM_APPLY_LAUNCH
    FEM_LAUNCH(k_apply_gather, (int)((P->N + 255) / 256), 256, 0, s, P->N, P->inc_ptr,
               reinterpret_cast<const float2*>(T.pk), u, isbd, y);
    return FEM_OK;
  }
  if (T.fused) {
    // one cooperative launch: as many CTAs as are resident at once, counters zeroed in-stream
    const int smem = tile_fused_smem(T, D);
    if (smem == 0) return set_error(FEM_ERR_STATE, "the fused tile launch does not fit this mesh");
    int* ctr = P->work_counter + 1;
    FEM_CUDA(cudaMemsetAsync(ctr, 0, 3 * sizeof(int), s));
    const void* fn = nullptr;
    const char* name = nullptr;
#define FEM_FUSED_PICK(DD, TT, PWT)                                   \
  do {                                                                \
    fn = (const void*)k_tiles_fused<DD, TT, PWT>;                     \
    name = "(k_tiles_fused<" #DD ", " #TT ">)";                       \
  } while (0)
    if (D == 2) {
      if (T.TE == 128) FEM_FUSED_PICK(2, 128, uint16_t);
      else FEM_FUSED_PICK(2, 256, uint16_t);
    } else {
      if (T.TE == 128) FEM_FUSED_PICK(3, 128, uint32_t);
      else FEM_FUSED_PICK(3, 256, uint32_t);
    }
#undef FEM_FUSED_PICK
    FEM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, nsm = 0, dev = 0;
    FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T.TE, smem));
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return set_error(FEM_ERR_STATE, "the fused tile kernel cannot be resident");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(per_sm * nsm));
    cfg.blockDim = dim3((unsigned)T.TE);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&a, (void*)&g, (void*)&node, (void*)&k, (void*)&f_kind, (void*)&f_arg,
                    (void*)&val, (void*)&b, (void*)&tab, (void*)&ctr, (void*)&err};
    const bool tm = g_timing.load(std::memory_order_relaxed);
    if (tm) timing_mark(name, s, true);
    FEM_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (tm) timing_mark(name, s, false);
    return FEM_OK;
  }
  const int smem = tile_smem_need(T, D, f_kind == FEM_F_SINPROD && want_b);
#define FEM_TILE_LAUNCH_K(KERNEL, TT)                                                                         \
  do {                                                                                                        \
    if (smem > 48 * 1024)                                                                                     \
      FEM_CUDA(cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));             \
    FEM_LAUNCH(KERNEL, T.ntiles, TT, smem, s, a, node, k, f_kind, f_arg, want_a, want_b, tab, err);         \
  } while (0)
  const bool sine3 = D == 3 && f_kind == FEM_F_SINPROD && want_b;
  if (D == 2) {
    if (T.TE == 128) FEM_TILE_LAUNCH_K((k_tile_elements<2, 128>), 128);
    else FEM_TILE_LAUNCH_K((k_tile_elements<2, 256>), 256);
  } else if (!sine3) {
    if (T.TE == 128) FEM_TILE_LAUNCH_K((k_tile_elements<3, 128>), 128);
    else FEM_TILE_LAUNCH_K((k_tile_elements<3, 256>), 256);
  } else {
    if (T.TE == 128) FEM_TILE_LAUNCH_K((k_tile_elements<3, 128, 6>), 128);
    else FEM_TILE_LAUNCH_K((k_tile_elements<3, 256, 6>), 256);
  }
#undef FEM_TILE_LAUNCH_K
  const int wpc = gather_warps(g.max_row);
  const int bt = 32 * wpc;
  const int gsm = wpc * gather_warp_bytes(g.max_row);
  const int64_t grid = (P->N + bt - 1) / bt;
  if (D == 2) {
    FEM_CUDA(cudaFuncSetAttribute(k_row_gather<2, uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm));
    // a third of the unified L1/shared storage as shared memory: fewer resident warps, but the L1 keeps
    // a row's packet sectors until its next packets are read (measured with three packets in flight per
    // thread: 0.187 ms, against 0.195 at a quarter or a sixth, 0.190 at a half, 0.194 at two thirds)
    FEM_CUDA(cudaFuncSetAttribute(k_row_gather<2, uint16_t>, cudaFuncAttributePreferredSharedMemoryCarveout, 33));
    FEM_LAUNCH((k_row_gather<2, uint16_t>), (int)grid, bt, gsm, s, g, val, b);
  } else {
    FEM_CUDA(cudaFuncSetAttribute(k_row_gather<3, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm));
    FEM_LAUNCH((k_row_gather<3, uint32_t>), (int)grid, bt, gsm, s, g, val, b);
  }
  return FEM_OK;
}

}  // namespace fem
