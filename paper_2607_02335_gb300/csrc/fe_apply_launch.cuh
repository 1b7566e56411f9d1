// fe_apply_launch.cuh -- host launchers of the apply kernels for one arithmetic V.
#pragma once
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "fe_recompute.cuh"

template <class V>
V fe_cast(double v);
template <>
inline double fe_cast<double>(double v) { return v; }
template <>
inline float fe_cast<float>(double v) { return (float)v; }
template <>
inline dw fe_cast<dw>(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
template <>
inline bfv fe_cast<bfv>(double v) {  // round to nearest even bf16
  return {__bfloat162float(__float2bfloat16_rn((float)v))};
}
template <>
inline hfv fe_cast<hfv>(double v) {
  return {__half2float(__float2half_rn((float)v))};
}

// even-odd form of M (tr: of M^T), from the FP64 tables
template <int N, class V>
void fill_eo(EO<N, V>& e, const double (&M0)[FE_MAXN][FE_MAXN], bool tr) {
  auto M = [&](int q, int r) { return tr ? M0[r][q] : M0[q][r]; };
  constexpr int H = N / 2, mid = N / 2;
  std::memset(&e, 0, sizeof(e));
  for (int q = 0; q < H; ++q) {
    for (int r = 0; r < H; ++r) {
      e.A[q][r] = fe_cast<V>(0.5 * (M(q, r) + M(q, N - 1 - r)));
      e.B[q][r] = fe_cast<V>(0.5 * (M(q, r) - M(q, N - 1 - r)));
    }
    if (N & 1) {
      e.cm[q] = fe_cast<V>(M(q, mid));
      e.cr[q] = fe_cast<V>(M(mid, q));
    }
  }
  if (N & 1) e.mm = fe_cast<V>(M(mid, mid));
}

// even-odd form of B' (EOB in fe_arith.h) from B = Dh: B'[q][s] = sum_{r > s} Dh[q][r]
template <int N, class V>
void fill_eob(EOB<N, V>& e, const HostTab& h) {
  using E = EOB<N, V>;
  double Bp[FE_MAXN][FE_MAXN] = {};
  for (int q = 0; q < N; ++q)
    for (int s = 0; s < N - 1; ++s) {
      double acc = 0.0;
      for (int r = s + 1; r < N; ++r) acc += h.Dh[q][r];
      Bp[q][s] = acc;
    }
  std::memset(&e, 0, sizeof(e));
  for (int q = 0; q < E::HO; ++q) {
    for (int s = 0; s < E::HI; ++s) {
      e.A[q][s] = fe_cast<V>(0.5 * (Bp[q][s] + Bp[q][E::NI - 1 - s]));
      e.B[q][s] = fe_cast<V>(0.5 * (Bp[q][s] - Bp[q][E::NI - 1 - s]));
    }
    if (E::NI & 1) e.cm[q] = fe_cast<V>(Bp[q][E::NI / 2]);
  }
  if (N & 1)
    for (int s = 0; s < E::HI; ++s) e.cr[s] = fe_cast<V>(Bp[N / 2][s]);
}

template <int N, class V>
Tab1D<N, V> make_tab(const HostTab& h) {
  Tab1D<N, V> t;
  for (int a = 0; a < N; ++a) {
    t.W_[a] = fe_cast<V>(h.w[a]);
    for (int b = 0; b < N; ++b) {
      t.V_[a][b] = fe_cast<V>(h.V[a][b]);
      t.D_[a][b] = fe_cast<V>(h.D[a][b]);
    }
  }
  fill_eo<N, V>(t.eV, h.V, false);
  fill_eo<N, V>(t.eVT, h.V, true);
  fill_eo<N, V>(t.eD, h.D, false);
  fill_eo<N, V>(t.eDT, h.D, true);
  fill_eob<N, V>(t.eB, h);
  return t;
}

template <int N, class V, int OP, int GEOM, int MODE = MODE_CELLS>
static fe_status launch_one(const ApplyArgs<N, V>& a, cudaStream_t st) {
  using C = Cfg<N>;
  const size_t smem = apply_smem_bytes<N, V>(OP);
  auto kern = [] {
    if constexpr (MODE == MODE_BRICKZ)
      return k_apply_zcarry<N, V, OP, GEOM>;
    else
      return k_apply<N, V, OP, GEOM, MODE>;
  }();
  static bool attr_done[64] = {};  // one attribute call per instantiation and device
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "apply smem attribute");
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
  }
  long long blocks;
  int threads = C::THREADS;
  if constexpr (MODE == MODE_BRICK) {
    constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
    blocks = (long long)((a.c.mx + BX - 1) / BX) * ((a.c.my + BY - 1) / BY) * a.c.mz;
    threads = BX * BY * C::N2;
  } else if constexpr (MODE == MODE_BRICKZ) {
    constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
    blocks = (long long)((a.c.mx + BX - 1) / BX) * ((a.c.my + BY - 1) / BY) *
             ((a.c.mz + a.zchunk - 1) / a.zchunk);
    threads = BX * BY * C::N2;
  } else if constexpr (MODE == MODE_PACKED) {
    blocks = (a.c.ncells / 8 + Packed<N>::UPB - 1) / Packed<N>::UPB;
  } else {
    blocks = (a.c.ncells - a.c.cell_base + C::CPB - 1) / C::CPB;
  }
  if (blocks > 0) kern<<<(unsigned)blocks, threads, smem, st>>>(a);
  return fe_cuda_check(cudaGetLastError(), "apply kernel launch");
}

// Recompute mode: per chunk of cells, the metric into the L2-sized scratch, then the stored-metric
// apply on the chunk.
template <int N, class V, int OP>
static fe_status launch_recompute(ApplyArgs<N, V> a, const ApplyLaunch& L,
                                  const typename NT<V>::GV* xyz, typename NT<V>::GV* scratch) {
  const fe_mesh* m = L.m;
  if (!xyz || !scratch) {
    fe_set_error("apply: recompute-mode buffers missing for this arithmetic");
    return FE_ERR_INVALID;
  }
  using G = GeoCfg<N>;
  const long long chunk = fe_rc_chunk_cells(N, m->ncells, sizeof(typename NT<V>::GV));
  RecomputeArgs<N, V> r;
  std::memset(&r, 0, sizeof(r));
  r.xyz = xyz;
  r.geo = scratch;
  r.skip = L.skip;
  r.tab = a.tab;
  a.c.geo = scratch;
  for (long long c0 = 0; c0 < m->ncells; c0 += chunk) {
    const long long c1 = c0 + chunk < m->ncells ? c0 + chunk : m->ncells;
    r.cell0 = c0;
    r.cell_end = c1;
    const long long gblocks = (c1 - c0 + G::CPB - 1) / G::CPB;
    k_recompute<N, V, OP>
        <<<(unsigned)gblocks, G::THREADS, recompute_smem_bytes<N, V>(), L.st>>>(r);
    FE_CUDA(cudaGetLastError(), "recompute kernel launch");
    a.c.cell_base = c0;
    a.c.geo_cell0 = c0;
    a.c.ncells = c1;
    FE_TRY((launch_one<N, V, OP, GEOM_STORED_K>(a, L.st)));
  }
  return FE_OK;
}

// the kernel of (operator, geometry mode); 16-bit operand types have stored geometry only
#ifndef FE_ZCARRY_MAXZ
#define FE_ZCARRY_MAXZ 16
#endif
// Layers per CTA of a z-carry launch (< 2: use the one-layer brick kernel).  The CTAs run
// zchunk layers each, so the grid's last wave decides the tail: the largest zchunk <=
// FE_ZCARRY_MAXZ whose grid fills at least four waves of resident CTAs, the last one to 97%
// (Q3 96^3, double-word: 15 layers for the Laplace kernel at 3 CTAs per SM, 9 for mass at 6).
template <int N, class V, int OP, int GEOM>
static fe_status zcarry_slots(int* slots) {
  static int cached[64] = {};
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev >= 0 && dev < 64 && cached[dev] > 0) {
    *slots = cached[dev];
    return FE_OK;
  }
  auto kern = k_apply_zcarry<N, V, OP, GEOM>;
  const size_t smem = apply_smem_bytes<N, V>(OP);
  FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
          "apply smem attribute");
  int per_sm = 0, sms = 0;
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
              &per_sm, kern, Brick<N>::BX * Brick<N>::BY * Cfg<N>::N2, smem),
          "occupancy");
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  *slots = per_sm * sms;
  if (dev >= 0 && dev < 64) cached[dev] = *slots;
  return FE_OK;
}

template <int N, class V>
static fe_status zcarry_chunk(const fe_mesh* m, int op, bool affine, int* zc) {
  int slots = 0;
  if (affine)
    FE_TRY((op == FE_LAPLACE ? zcarry_slots<N, V, FE_LAPLACE, GEOM_AFFINE_K>(&slots)
                             : zcarry_slots<N, V, FE_MASS, GEOM_AFFINE_K>(&slots)));
  else
    FE_TRY((op == FE_LAPLACE ? zcarry_slots<N, V, FE_LAPLACE, GEOM_STORED_K>(&slots)
                             : zcarry_slots<N, V, FE_MASS, GEOM_STORED_K>(&slots)));
  *zc = 0;
  // FE_ZCARRY_CHUNK=k in the environment forces k layers per CTA (0 or 1: the one-layer kernel)
  if (const char* force = std::getenv("FE_ZCARRY_CHUNK")) {
    const int k = std::atoi(force);
    *zc = k < 2 ? 0 : (k < m->d.mz ? k : m->d.mz);
    return FE_OK;
  }
  if (slots < 1) return FE_OK;
  constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
  const double per_layer = (double)((m->d.mx + BX - 1) / BX) * ((m->d.my + BY - 1) / BY);
  for (int z = FE_ZCARRY_MAXZ < m->d.mz ? FE_ZCARRY_MAXZ : m->d.mz; z >= 2; --z) {
    const double waves = (double)((m->d.mz + z - 1) / z) * per_layer / slots;
    if (waves >= 4.0 && waves / std::ceil(waves) >= 0.97) {
      *zc = z;
      break;
    }
  }
  return FE_OK;
}

template <int N, class V, int MODE>
static fe_status launch_geom(const ApplyArgs<N, V>& a, int op, bool affine, cudaStream_t st) {
  if constexpr (!NT<V>::LOWP) {
    if (affine)
      return op == FE_LAPLACE ? launch_one<N, V, FE_LAPLACE, GEOM_AFFINE_K, MODE>(a, st)
                              : launch_one<N, V, FE_MASS, GEOM_AFFINE_K, MODE>(a, st);
  }
  return op == FE_LAPLACE ? launch_one<N, V, FE_LAPLACE, GEOM_STORED_K, MODE>(a, st)
                          : launch_one<N, V, FE_MASS, GEOM_STORED_K, MODE>(a, st);
}

template <int N, class V>
static fe_status launch_apply_n(const ApplyLaunch& L, const typename NT<V>::GV* geo,
                                const typename NT<V>::GV* xyz, typename NT<V>::GV* scratch) {
  const fe_mesh* m = L.m;
  ApplyArgs<N, V> a;
  std::memset(&a, 0, sizeof(a));
  a.c.x = static_cast<const typename NT<V>::SV*>(L.x);
  a.c.y = static_cast<typename NT<V>::SV*>(L.y);
  a.c.geo = geo;
  a.c.ncells = m->ncells;
  a.c.mx = m->d.mx;
  a.c.my = m->d.my;
  a.c.mz = m->d.mz;
  a.c.dirichlet = fe_dir_mask(m);
  a.skip = L.skip;
  const double hx = 1.0 / m->d.mx, hy = 1.0 / m->d.my, hz = 1.0 / fe_mz_global(m),
               det = hx * hy * hz;
  a.c.aff[0] = fe_cast<V>(det / (hx * hx));
  a.c.aff[1] = fe_cast<V>(det / (hy * hy));
  a.c.aff[2] = fe_cast<V>(det / (hz * hz));
  a.c.aff[3] = fe_cast<V>(det);
  a.tab = make_tab<N, V>(m->tab);
  a.c.oscale = 1.0f;
  if constexpr (NT<V>::LOWP) {
    if (m->d.geom_mode != FE_GEOM_STORED || !geo) {
      fe_set_error("apply: 16-bit contractions need stored geometry");
      return FE_ERR_INVALID;
    }
    a.c.oscale = 1.0f / m->gscale[L.op == FE_LAPLACE ? 0 : 1];
  }
  constexpr int PREC = sizeof(typename NT<V>::SV) == 8 ? FE_F64 : FE_F32;
  if constexpr (!NT<V>::LOWP) {
    if (m->d.geom_mode == FE_GEOM_RECOMPUTE) {
      FE_TRY((L.op == FE_LAPLACE ? launch_recompute<N, V, FE_LAPLACE>(a, L, xyz, scratch)
                                 : launch_recompute<N, V, FE_MASS>(a, L, xyz, scratch)));
      if (L.assemble && L.brick_out) {
        L.brick_out[0] = L.brick_out[1] = 1;
        return FE_OK;
      }
      return L.assemble ? fe_launch_dss(m, PREC, L.y, L.st) : FE_OK;
    }
  }
  const bool affine = m->d.geom_mode == FE_GEOM_AFFINE;
  if (m->packed) {  // 2^3-packed storage units: unit-internal assembly in the kernel
    if constexpr (N < FE_ROLL_MINN && N <= 4) {
      FE_TRY((launch_geom<N, V, MODE_PACKED>(a, L.op, affine, L.st)));
      if (!L.assemble) return FE_OK;
      if (L.brick_out) {
        L.brick_out[0] = L.brick_out[1] = 1;
        return FE_OK;
      }
      return fe_launch_dss(m, PREC, L.y, L.st);
    } else {
      fe_set_error("apply: packed storage units are provided for degrees 1 to 3");
      return FE_ERR_INVALID;
    }
  }
// Assembled applies sum the intra-brick interfaces in the kernel up to n = FE_FUSE_MAXN.  Above it
// the bricks hold fewer cells than the unfused tile (n = 6, 7) or the kernel needs more
// registers, and the measured assembled time was no better than apply + full DSS.
#ifndef FE_FUSE_MAXN
#define FE_FUSE_MAXN 4
#endif
  const bool fuse = L.assemble && N <= FE_FUSE_MAXN;
  // Fused assembled applies with the DSS passes left to this launcher also sum the z-interfaces
  // in the kernel: a CTA walks zchunk layers of its brick column; only the interfaces between
  // chunks remain for the z-pass.
  if constexpr (N <= FE_FUSE_MAXN && N < FE_ROLL_MINN && !NT<V>::LOWP) {
    if (fuse && !L.brick_out) {
      int zc = 0;
      FE_TRY((zcarry_chunk<N, V>(m, L.op, affine, &zc)));
      if (zc >= 2) {
        a.zchunk = zc;
        FE_TRY((launch_geom<N, V, MODE_BRICKZ>(a, L.op, affine, L.st)));
        return fe_launch_dss_strided3(m, PREC, L.y, Brick<N>::BX, Brick<N>::BY, zc, L.st);
      }
    }
  }
  if (fuse)
    FE_TRY((launch_geom<N, V, MODE_BRICK>(a, L.op, affine, L.st)));
  else
    FE_TRY((launch_geom<N, V, MODE_CELLS>(a, L.op, affine, L.st)));
  if (!L.assemble) return FE_OK;
  if (L.brick_out) {  // the caller runs the passes (one launch over many blocks)
    L.brick_out[0] = fuse ? Brick<N>::BX : 1;
    L.brick_out[1] = fuse ? Brick<N>::BY : 1;
    return FE_OK;
  }
  return fuse ? fe_launch_dss_strided(m, PREC, L.y, Brick<N>::BX, Brick<N>::BY, L.st)
              : fe_launch_dss(m, PREC, L.y, L.st);
}

template <class V>
static fe_status launch_apply_v(const ApplyLaunch& L, const typename NT<V>::GV* geo,
                                const typename NT<V>::GV* xyz, typename NT<V>::GV* scratch) {
  switch (L.m->n) {
    case 2: return launch_apply_n<2, V>(L, geo, xyz, scratch);
    case 3: return launch_apply_n<3, V>(L, geo, xyz, scratch);
    case 4: return launch_apply_n<4, V>(L, geo, xyz, scratch);
    case 5: return launch_apply_n<5, V>(L, geo, xyz, scratch);
    case 6: return launch_apply_n<6, V>(L, geo, xyz, scratch);
    case 7: return launch_apply_n<7, V>(L, geo, xyz, scratch);
    case 8: return launch_apply_n<8, V>(L, geo, xyz, scratch);
  }
  fe_set_error("apply: unsupported n = %d", L.m->n);
  return FE_ERR_INVALID;
}
