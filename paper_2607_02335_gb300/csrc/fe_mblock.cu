// fe_mblock.cu -- block-structured meshes: topology builder and the inter-block summation
// (Sec. 4.2 "Generalization to Block-Structured Grids", Algorithm "Unstructured Inter-Block
// Summation").
//
// Every block is an ordinary structured mesh (its own fe_mesh with a trilinear geometry), so the
// volumetric apply and the structured DSS inside a block are the single-block kernels run on the
// block's slice of the cell-wise vector.  What is new is the summation across block interfaces,
// split by codimension into three disjoint node sets:
//   faces    -- the nodes strictly inside a macro-face shared by two blocks: for every pair of
//               matching cell faces, the two copies are summed and written back to both (side b
//               re-indexed into side a's frame by a 3-bit orientation: swap, flip s, flip t);
//               nodes on cell edges inside the face have two copies per side, but the structured
//               pass already made them equal, so each cell-face pair still adds exactly A + B;
//   lines    -- the nodes strictly inside a macro-edge (any number of blocks): one thread per
//               node sums one representative copy per block and writes every copy;
//   vertices -- the macro-corners, likewise.
// The structured pass has replicated the within-block sum on every within-block copy, so adding
// one representative per block gives the assembled value.  The three sets are disjoint, so the
// launches need no atomics and can run in any order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "fe_vec.cuh"

namespace {

// face pair: side a and side b (block cell offsets, dims, face id), orientation of b vs a
struct MbFace {
  long long offa, offb;  // first cell of the blocks
  int da[3], db[3];      // cells per direction of the blocks
  int fa, fb;            // local face: 2*axis + side
  int orient;            // bit 0 swap, bit 1 flip s', bit 2 flip t'
};

// one block's local face f: the axis, the side, and the two tangent axes (increasing order)
__host__ __device__ inline void face_axes(int f, int* axis, int* side, int* t1, int* t2) {
  *axis = f >> 1;
  *side = f & 1;
  *t1 = *axis == 0 ? 1 : 0;
  *t2 = *axis == 2 ? 1 : 2;
}

// Work item e of face pair F (cell face (cu, cv) of side a and node (aa, bb) on it): false for
// nodes on the macro-face boundary (left to lines and vertices), else the cell-wise indices of
// the two copies (-1 if an index falls outside its block, which the builder rules out).
__host__ __device__ inline bool face_map(const MbFace& F, int n, long long e, long long* ia,
                                         long long* ib) {
  const int p = n - 1;
  int axa, sda, t1a, t2a, axb, sdb, t1b, t2b;
  face_axes(F.fa, &axa, &sda, &t1a, &t2a);
  face_axes(F.fb, &axb, &sdb, &t1b, &t2b);
  const int cu_n = F.da[t1a];
  const int N1a = cu_n * p, N2a = F.da[t2a] * p;
  const int N1b = F.db[t1b] * p, N2b = F.db[t2b] * p;
  const bool swap = F.orient & 1, fs = F.orient & 2, ft = F.orient & 4;
  const int aa = (int)(e % n), bb = (int)((e / n) % n);
  const long long cf = e / (n * n);
  const int cu = (int)(cf % cu_n), cv = (int)(cf / cu_n);
  const int s = cu * p + aa, t = cv * p + bb;
  if (s == 0 || s == N1a || t == 0 || t == N2a) return false;
  int ca[3], la[3];
  ca[axa] = sda ? F.da[axa] - 1 : 0;
  la[axa] = sda ? p : 0;
  ca[t1a] = cu;
  la[t1a] = aa;
  ca[t2a] = cv;
  la[t2a] = bb;
  // side b: the node and the cell-face centre (doubled coordinates) through the orientation
  const int sc2 = 2 * cu * p + p, tc2 = 2 * cv * p + p;
  int sb, tb, sbc2, tbc2;
  if (!swap) {
    sb = fs ? N1b - s : s;
    tb = ft ? N2b - t : t;
    sbc2 = fs ? 2 * N1b - sc2 : sc2;
    tbc2 = ft ? 2 * N2b - tc2 : tc2;
  } else {
    sb = fs ? N1b - t : t;
    tb = ft ? N2b - s : s;
    sbc2 = fs ? 2 * N1b - tc2 : tc2;
    tbc2 = ft ? 2 * N2b - sc2 : sc2;
  }
  const int cub = (sbc2 - p) / (2 * p), cvb = (tbc2 - p) / (2 * p);
  int cb[3], lb[3];
  cb[axb] = sdb ? F.db[axb] - 1 : 0;
  lb[axb] = sdb ? p : 0;
  cb[t1b] = cub;
  lb[t1b] = sb - cub * p;
  cb[t2b] = cvb;
  lb[t2b] = tb - cvb * p;
  bool ok = true;
  for (int k = 0; k < 3; ++k)
    ok = ok && cb[k] >= 0 && cb[k] < F.db[k] && lb[k] >= 0 && lb[k] <= p;
  const long long n3 = (long long)n * n * n;
  *ia = (F.offa + ((long long)ca[2] * F.da[1] + ca[1]) * F.da[0] + ca[0]) * n3 +
        ((long long)la[2] * n + la[1]) * n + la[0];
  *ib = ok ? (F.offb + ((long long)cb[2] * F.db[1] + cb[1]) * F.db[0] + cb[0]) * n3 +
                 ((long long)lb[2] * n + lb[1]) * n + lb[0]
           : -1;
  return true;
}

template <class S>
__global__ void k_mb_faces(S* __restrict__ v, const MbFace* __restrict__ faces, int n) {
  const MbFace F = faces[blockIdx.y];
  int ax, sd, t1, t2;
  face_axes(F.fa, &ax, &sd, &t1, &t2);
  const long long items = (long long)F.da[t1] * F.da[t2] * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < items;
       e += (long long)gridDim.x * blockDim.x) {
    long long ia, ib;
    if (!face_map(F, n, e, &ia, &ib) || ib < 0) continue;
    const S sum = v[ia] + v[ib];
    v[ia] = sum;
    v[ib] = sum;
  }
}

// lines and vertices: one entity per thread; reps[e*R + r] one copy per sharing block (-1 pad),
// copies[e*C + c] every copy (-1 pad)
template <class S>
__global__ void k_mb_entities(S* __restrict__ v, const long long* __restrict__ reps, int R,
                              const long long* __restrict__ copies, int C, long long nent) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nent;
       e += (long long)gridDim.x * blockDim.x) {
    S sum = 0;
    for (int r = 0; r < R; ++r) {
      const long long i = reps[e * R + r];
      if (i >= 0) sum += v[i];
    }
    for (int c = 0; c < C; ++c) {
      const long long i = copies[e * C + c];
      if (i >= 0) v[i] = sum;
    }
  }
}

unsigned grid_cap(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

struct fe_mbmesh {
  int nblocks = 0, p = 0, n = 0, device = 0;
  std::vector<fe_mesh*> blocks;
  std::vector<long long> off;  // first cell of every block
  long long ncells = 0, ncw = 0, nu = 0;
  MbFace* faces = nullptr;     // device
  int nfaces = 0;
  long long max_face_items = 0;
  long long *reps = nullptr, *copies = nullptr;  // device
  int R = 0, C = 0;
  long long nent = 0, nedge_ent = 0;
  int nvert_ent = 0, max_valence = 0;
};

namespace {

// corner of block-local face f at face-local (u, v)
int face_corner(int f, int u, int v) {
  int axis, side, t1, t2;
  face_axes(f, &axis, &side, &t1, &t2);
  return (side << axis) | (u << t1) | (v << t2);
}

void free_mb(fe_mbmesh* M) {
  for (fe_mesh* b : M->blocks)
    if (b) fe_mesh_destroy(b);
  cudaFree(M->faces);
  cudaFree(M->reps);
  cudaFree(M->copies);
  delete M;
}

struct Copy {
  long long idx;
  int block;
};

}  // namespace

extern "C" fe_status fe_mb_create(const fe_mb_desc* d, void* stream, fe_mbmesh** out) {
  if (!d || !out || !d->dims || !d->block_verts || !d->vxyz) {
    fe_set_error("fe_mb_create: null argument");
    return FE_ERR_INVALID;
  }
  *out = nullptr;
  if (d->nblocks < 1 || d->nverts < 1 || d->degree < 1 || d->degree > 7) {
    fe_set_error("fe_mb_create: bad sizes (nblocks %d, nverts %d, degree %d)", d->nblocks,
                 d->nverts, d->degree);
    return FE_ERR_INVALID;
  }
  const int nb = d->nblocks, p = d->degree, n = p + 1;
  for (int b = 0; b < nb; ++b) {
    for (int a = 0; a < 3; ++a)
      if (d->dims[3 * b + a] < 1) {
        fe_set_error("fe_mb_create: block %d has a non-positive cell count", b);
        return FE_ERR_INVALID;
      }
    for (int c = 0; c < 8; ++c)
      if (d->block_verts[8 * b + c] < 0 || d->block_verts[8 * b + c] >= d->nverts) {
        fe_set_error("fe_mb_create: block %d corner %d has a bad vertex number", b, c);
        return FE_ERR_INVALID;
      }
    // right-handed corner frame (the trilinear map's Jacobian at corner 0)
    const double* X0 = d->vxyz + 3 * d->block_verts[8 * b];
    double e[3][3];
    for (int k = 0; k < 3; ++k) {
      const double* Xk = d->vxyz + 3 * d->block_verts[8 * b + (1 << k)];
      for (int a = 0; a < 3; ++a) e[k][a] = Xk[a] - X0[a];
    }
    const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                       e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    if (!(det > 0.0)) {
      fe_set_error("fe_mb_create: block %d is left-handed or degenerate", b);
      return FE_ERR_INVALID;
    }
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(d->device), "cudaSetDevice");
  fe_mbmesh* M = new (std::nothrow) fe_mbmesh();
  if (!M) {
    fe_set_error("fe_mb_create: host allocation failed");
    return FE_ERR_OOM;
  }
  M->nblocks = nb;
  M->p = p;
  M->n = n;
  M->device = d->device;
  const long long n3 = (long long)n * n * n;
  for (int b = 0; b < nb; ++b) {
    M->off.push_back(M->ncells);
    M->ncells += (long long)d->dims[3 * b] * d->dims[3 * b + 1] * d->dims[3 * b + 2];
  }
  M->ncw = M->ncells * n3;

  // ---- faces: match by the sorted corner vertices
  std::map<std::vector<int>, std::vector<std::pair<int, int>>> fmap;  // key -> (block, face)
  for (int b = 0; b < nb; ++b)
    for (int f = 0; f < 6; ++f) {
      std::vector<int> key;
      for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) key.push_back(d->block_verts[8 * b + face_corner(f, u, v)]);
      std::sort(key.begin(), key.end());
      fmap[key].push_back({b, f});
    }
  std::vector<MbFace> hfaces;
  long long nu = 0;
  for (auto& kv : fmap) {
    auto& occ = kv.second;
    if (occ.size() > 2) {
      fe_set_error("fe_mb_create: a face is shared by more than two blocks");
      free_mb(M);
      return FE_ERR_INVALID;
    }
    int axis, side, t1, t2;
    face_axes(occ[0].second, &axis, &side, &t1, &t2);
    const int* da = d->dims + 3 * occ[0].first;
    nu += (long long)(da[t1] * p - 1) * (da[t2] * p - 1);  // open face interior, counted once
    if (occ.size() < 2) continue;
    const int a = occ[0].first, fa = occ[0].second, b = occ[1].first, fb = occ[1].second;
    // where a's face corners (0,0), (1,0), (0,1) sit on b's face
    auto pos_on_b = [&](int vid, int* u, int* v) {
      for (int uu = 0; uu < 2; ++uu)
        for (int vv = 0; vv < 2; ++vv)
          if (d->block_verts[8 * b + face_corner(fb, uu, vv)] == vid) {
            *u = uu;
            *v = vv;
            return true;
          }
      return false;
    };
    int u0, v0, u1, v1, u2, v2;
    bool ok = pos_on_b(d->block_verts[8 * a + face_corner(fa, 0, 0)], &u0, &v0) &&
              pos_on_b(d->block_verts[8 * a + face_corner(fa, 1, 0)], &u1, &v1) &&
              pos_on_b(d->block_verts[8 * a + face_corner(fa, 0, 1)], &u2, &v2);
    MbFace F;
    std::memset(&F, 0, sizeof(F));
    F.offa = M->off[a];
    F.offb = M->off[b];
    for (int k = 0; k < 3; ++k) {
      F.da[k] = d->dims[3 * a + k];
      F.db[k] = d->dims[3 * b + k];
    }
    F.fa = fa;
    F.fb = fb;
    const bool swap = (u1 == u0);  // a's s runs along b's t
    const bool flip_s = swap ? (u2 < u0) : (u1 < u0);
    const bool flip_t = swap ? (v1 < v0) : (v2 < v0);
    F.orient = (swap ? 1 : 0) | (flip_s ? 2 : 0) | (flip_t ? 4 : 0);
    int axb, sdb, t1b, t2b;
    face_axes(fb, &axb, &sdb, &t1b, &t2b);
    const int Na1 = F.da[t1] * p, Na2 = F.da[t2] * p;
    const int Nb1 = F.db[t1b] * p, Nb2 = F.db[t2b] * p;
    if (!ok || (!swap && (Na1 != Nb1 || Na2 != Nb2)) || (swap && (Na1 != Nb2 || Na2 != Nb1))) {
      fe_set_error("fe_mb_create: blocks %d and %d do not conform on their shared face", a, b);
      free_mb(M);
      return FE_ERR_INVALID;
    }
    hfaces.push_back(F);
    M->max_face_items = std::max(M->max_face_items, (long long)F.da[t1] * F.da[t2] * n * n);
  }

  // ---- edges: group by the sorted end vertices; nodes strictly inside each shared edge
  struct EdgeOcc {
    int block, axis, s1, s2;
    bool reversed;
  };
  std::map<std::pair<int, int>, std::vector<EdgeOcc>> emap;
  for (int b = 0; b < nb; ++b)
    for (int axis = 0; axis < 3; ++axis) {
      const int e1 = axis == 0 ? 1 : 0, e2 = axis == 2 ? 1 : 2;
      for (int s1 = 0; s1 < 2; ++s1)
        for (int s2 = 0; s2 < 2; ++s2) {
          const int clo = (s1 << e1) | (s2 << e2), chi = clo | (1 << axis);
          const int vlo = d->block_verts[8 * b + clo], vhi = d->block_verts[8 * b + chi];
          emap[{std::min(vlo, vhi), std::max(vlo, vhi)}].push_back({b, axis, s1, s2, vlo > vhi});
        }
    }
  std::vector<std::vector<Copy>> ent_copies;  // per entity: every copy
  for (auto& kv : emap) {
    auto& occ = kv.second;
    const int N = d->dims[3 * occ[0].block + occ[0].axis] * p;
    nu += N - 1;
    if (occ.size() < 2) continue;
    for (auto& o : occ)
      if (d->dims[3 * o.block + o.axis] * p != N) {
        fe_set_error("fe_mb_create: blocks do not conform on a shared edge");
        free_mb(M);
        return FE_ERR_INVALID;
      }
    for (int q = 1; q < N; ++q) {
      std::vector<Copy> cp;
      for (auto& o : occ) {
        const int e1 = o.axis == 0 ? 1 : 0, e2 = o.axis == 2 ? 1 : 2;
        const int* db = d->dims + 3 * o.block;
        const int ql = o.reversed ? N - q : q;
        int c[3], l[3];
        c[e1] = o.s1 ? db[e1] - 1 : 0;
        l[e1] = o.s1 ? p : 0;
        c[e2] = o.s2 ? db[e2] - 1 : 0;
        l[e2] = o.s2 ? p : 0;
        auto push = [&](int cell, int loc) {
          c[o.axis] = cell;
          l[o.axis] = loc;
          const long long idx = (M->off[o.block] + ((long long)c[2] * db[1] + c[1]) * db[0] + c[0]) * n3 +
                                ((long long)l[2] * n + l[1]) * n + l[0];
          cp.push_back({idx, o.block});
        };
        if (ql % p == 0) {  // on a cell vertex: two cells of this block along the edge
          push(ql / p - 1, p);
          push(ql / p, 0);
        } else {
          push(ql / p, ql % p);
        }
      }
      ent_copies.push_back(cp);
    }
  }
  M->nedge_ent = (long long)ent_copies.size();

  // ---- vertices: group the block corners by vertex number
  std::map<int, std::vector<std::pair<int, int>>> vmap;  // vertex -> (block, corner)
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < 8; ++c) vmap[d->block_verts[8 * b + c]].push_back({b, c});
  for (auto& kv : vmap) {
    nu += 1;
    if (kv.second.size() < 2) continue;
    std::vector<Copy> cp;
    for (auto& bc : kv.second) {
      const int b = bc.first, c = bc.second;
      const int* db = d->dims + 3 * b;
      int cc[3], l[3];
      for (int a = 0; a < 3; ++a) {
        const int s = (c >> a) & 1;
        cc[a] = s ? db[a] - 1 : 0;
        l[a] = s ? p : 0;
      }
      cp.push_back({(M->off[b] + ((long long)cc[2] * db[1] + cc[1]) * db[0] + cc[0]) * n3 +
                        ((long long)l[2] * n + l[1]) * n + l[0],
                    b});
    }
    ent_copies.push_back(cp);
    ++M->nvert_ent;
  }
  // block interiors
  for (int b = 0; b < nb; ++b)
    nu += (long long)(d->dims[3 * b] * p - 1) * (d->dims[3 * b + 1] * p - 1) *
          (d->dims[3 * b + 2] * p - 1);
  M->nu = nu;

  // ---- padded sharing lists: one representative per block, and every copy
  M->nent = (long long)ent_copies.size();
  for (auto& cp : ent_copies) {
    std::vector<int> bl;
    for (auto& c : cp)
      if (std::find(bl.begin(), bl.end(), c.block) == bl.end()) bl.push_back(c.block);
    M->R = std::max(M->R, (int)bl.size());
    M->C = std::max(M->C, (int)cp.size());
  }
  M->max_valence = M->R;
  std::vector<long long> hreps((size_t)M->nent * std::max(M->R, 1), -1),
      hcopies((size_t)M->nent * std::max(M->C, 1), -1);
  for (long long e = 0; e < M->nent; ++e) {
    auto& cp = ent_copies[(size_t)e];
    std::vector<int> seen;
    int r = 0;
    for (size_t c = 0; c < cp.size(); ++c) {
      hcopies[(size_t)e * M->C + c] = cp[c].idx;
      if (std::find(seen.begin(), seen.end(), cp[c].block) == seen.end()) {
        seen.push_back(cp[c].block);
        hreps[(size_t)e * M->R + r++] = cp[c].idx;
      }
    }
  }
  // ---- self-check on the host: both copies of every face item, and every copy of every line and
  // vertex entity, sit at the same physical point (trilinear block maps at the GLL nodes)
  {
    HostTab tab;
    fe_host_tables(p, &tab);
    auto node_xyz = [&](long long idx, double x[3]) {
      const long long cell = idx / n3;
      const int loc = (int)(idx - cell * n3);
      int b = (int)(std::upper_bound(M->off.begin(), M->off.end(), cell) - M->off.begin()) - 1;
      const int* db = d->dims + 3 * b;
      const long long c = cell - M->off[b];
      const int cx = (int)(c % db[0]), cy = (int)((c / db[0]) % db[1]),
                cz = (int)(c / ((long long)db[0] * db[1]));
      const double X[3] = {(cx + tab.t[loc % n]) / db[0], (cy + tab.t[(loc / n) % n]) / db[1],
                           (cz + tab.t[loc / (n * n)]) / db[2]};
      for (int a = 0; a < 3; ++a) x[a] = 0.0;
      for (int k = 0; k < 8; ++k) {
        const double w = ((k & 1) ? X[0] : 1.0 - X[0]) * ((k & 2) ? X[1] : 1.0 - X[1]) *
                         ((k & 4) ? X[2] : 1.0 - X[2]);
        for (int a = 0; a < 3; ++a) x[a] += w * d->vxyz[3 * d->block_verts[8 * b + k] + a];
      }
    };
    double scale = 0.0;
    for (int i = 0; i < 3 * d->nverts; ++i) scale = std::max(scale, std::fabs(d->vxyz[i]));
    const double tol = 1e-9 * (scale > 0.0 ? scale : 1.0);
    auto same = [&](long long i0, long long i1) {
      double x0[3], x1[3];
      node_xyz(i0, x0);
      node_xyz(i1, x1);
      return std::fabs(x0[0] - x1[0]) <= tol && std::fabs(x0[1] - x1[1]) <= tol &&
             std::fabs(x0[2] - x1[2]) <= tol;
    };
    bool good = true;
    for (const MbFace& F : hfaces) {
      int ax, sd, t1, t2;
      face_axes(F.fa, &ax, &sd, &t1, &t2);
      const long long items = (long long)F.da[t1] * F.da[t2] * n * n;
      for (long long e = 0; e < items && good; ++e) {
        long long ia, ib;
        if (face_map(F, n, e, &ia, &ib)) good = ib >= 0 && same(ia, ib);
      }
    }
    for (auto& cp : ent_copies)
      for (size_t c = 1; c < cp.size() && good; ++c) good = same(cp[0].idx, cp[c].idx);
    if (!good) {
      fe_set_error("fe_mb_create: interface nodes do not coincide (inconsistent macro-mesh)");
      free_mb(M);
      return FE_ERR_INVALID;
    }
  }

  fe_status s = FE_OK;
  M->nfaces = (int)hfaces.size();
  if (M->nfaces > 65535) {
    fe_set_error("fe_mb_create: more than 65535 shared faces");
    s = FE_ERR_INVALID;
  }
  if (s == FE_OK && M->nfaces) {
    s = fe_cuda_check(cudaMalloc((void**)&M->faces, hfaces.size() * sizeof(MbFace)), "mb faces");
    if (s == FE_OK)
      s = fe_cuda_check(cudaMemcpy(M->faces, hfaces.data(), hfaces.size() * sizeof(MbFace),
                                   cudaMemcpyHostToDevice), "mb faces");
  }
  if (s == FE_OK && M->nent) {
    s = fe_cuda_check(cudaMalloc((void**)&M->reps, hreps.size() * sizeof(long long)), "mb lists");
    if (s == FE_OK)
      s = fe_cuda_check(cudaMalloc((void**)&M->copies, hcopies.size() * sizeof(long long)), "mb lists");
    if (s == FE_OK)
      s = fe_cuda_check(cudaMemcpy(M->reps, hreps.data(), hreps.size() * sizeof(long long),
                                   cudaMemcpyHostToDevice), "mb lists");
    if (s == FE_OK)
      s = fe_cuda_check(cudaMemcpy(M->copies, hcopies.data(), hcopies.size() * sizeof(long long),
                                   cudaMemcpyHostToDevice), "mb lists");
  }
  // ---- one structured mesh per block, trilinear geometry
  for (int b = 0; b < nb && s == FE_OK; ++b) {
    fe_mesh_desc bd;
    std::memset(&bd, 0, sizeof(bd));
    bd.mx = d->dims[3 * b];
    bd.my = d->dims[3 * b + 1];
    bd.mz = d->dims[3 * b + 2];
    bd.degree = p;
    bd.geom_mode = FE_GEOM_STORED;
    bd.device = d->device;
    double corners[24];
    for (int c = 0; c < 8; ++c)
      for (int a = 0; a < 3; ++a) corners[3 * c + a] = d->vxyz[3 * d->block_verts[8 * b + c] + a];
    fe_mesh* bm = nullptr;
    s = fe_mesh_create_impl(&bd, corners, stream, &bm);
    M->blocks.push_back(bm);
  }
  if (s != FE_OK) {
    free_mb(M);
    return s;
  }
  *out = M;
  return FE_OK;
}

extern "C" fe_status fe_mb_destroy(fe_mbmesh* M) {
  if (!M) return FE_OK;
  FeDeviceGuard device_guard;
  device_guard.set(M->device);
  cudaDeviceSynchronize();
  free_mb(M);
  return FE_OK;
}

extern "C" fe_status fe_mb_layout(const fe_mbmesh* M, fe_layout* out) {
  if (!M || !out) {
    fe_set_error("fe_mb_layout: null argument");
    return FE_ERR_INVALID;
  }
  out->n_cells = M->ncells;
  out->nodes_per_cell = (long long)M->n * M->n * M->n;
  out->cellwise_len = M->ncw;
  out->unique_dofs = M->nu;
  out->layout_id = 0;
  return FE_OK;
}

extern "C" fe_status fe_mb_info(const fe_mbmesh* M, int* face_pairs, long long* edge_entities,
                                int* vertex_entities, int* max_valence) {
  if (!M) {
    fe_set_error("fe_mb_info: null mesh");
    return FE_ERR_INVALID;
  }
  if (face_pairs) *face_pairs = M->nfaces;
  if (edge_entities) *edge_entities = M->nedge_ent;
  if (vertex_entities) *vertex_entities = M->nvert_ent;
  if (max_valence) *max_valence = M->max_valence;
  return FE_OK;
}

// inter-block summation on an assembled-per-block vector
template <class S>
static fe_status interblock(const fe_mbmesh* M, S* v, cudaStream_t st) {
  if (M->nfaces) {
    dim3 grid(grid_cap(M->max_face_items, 256) > 64 ? 64 : grid_cap(M->max_face_items, 256),
              M->nfaces);
    k_mb_faces<S><<<grid, 256, 0, st>>>(v, M->faces, M->n);
  }
  if (M->nent)
    k_mb_entities<S><<<grid_cap(M->nent, 128), 128, 0, st>>>(v, M->reps, M->R, M->copies, M->C,
                                                               M->nent);
  return fe_cuda_check(cudaGetLastError(), "inter-block summation launch");
}

static fe_status mb_check(const fe_mbmesh* M, fe_prec prec, const void* a, const void* b,
                          const char* what) {
  if (!M || !a || !b) {
    fe_set_error("%s: null argument", what);
    return FE_ERR_INVALID;
  }
  if (!fe_aligned(a) || !fe_aligned(b)) {
    fe_set_error("%s: vectors must be 16-byte aligned", what);
    return FE_ERR_INVALID;
  }
  if (prec != FE_F64 && prec != FE_F32) {
    fe_set_error("%s: precision %d not provided (FE_F64, FE_F32)", what, (int)prec);
    return FE_ERR_INVALID;
  }
  return FE_OK;
}

extern "C" fe_status fe_mb_dss(const fe_mbmesh* M, fe_prec prec, const void* r, void* z,
                               void* stream) {
  FE_TRY(mb_check(M, prec, r, z, "fe_mb_dss"));
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(M->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = prec == FE_F64 ? sizeof(double) : sizeof(float);
  if (r != z)
    FE_CUDA(cudaMemcpyAsync(z, r, (size_t)M->ncw * es, cudaMemcpyDeviceToDevice, st), "mb dss copy");
  FE_TRY(fe_launch_dss_blocks(M->blocks.data(), M->off.data(), M->nblocks, prec, z, 1, 1, st));
  return prec == FE_F64 ? interblock<double>(M, (double*)z, st) : interblock<float>(M, (float*)z, st);
}

extern "C" fe_status fe_mb_apply(const fe_mbmesh* M, fe_op op, fe_prec prec, const void* x,
                                 void* y, unsigned flags, void* stream) {
  FE_TRY(mb_check(M, prec, x, y, "fe_mb_apply"));
  if (op != FE_LAPLACE && op != FE_MASS) {
    fe_set_error("fe_mb_apply: unknown operator %d", (int)op);
    return FE_ERR_INVALID;
  }
  if (flags & ~(FE_ASSEMBLE | FE_NATIVE_F64)) {
    fe_set_error("fe_mb_apply: unknown flags 0x%x", flags);
    return FE_ERR_INVALID;
  }
  const size_t es = prec == FE_F64 ? sizeof(double) : sizeof(float);
  const char *xb = (const char*)x, *yb = (const char*)y;
  if (xb < yb + M->ncw * es && yb < xb + M->ncw * es) {
    fe_set_error("fe_mb_apply: x and y overlap");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(M->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const bool native = (flags & FE_NATIVE_F64) && prec == FE_F64;
  const long long n3 = (long long)M->n * M->n * M->n;
  int brick[2] = {1, 1};
  for (int b = 0; b < M->nblocks; ++b) {
    const fe_mesh* bm = M->blocks[b];
    FE_TRY(fe_ensure_geometry(bm, prec, native));
    const size_t o = (size_t)M->off[b] * n3 * es;
    ApplyLaunch L{bm, (int)op, xb + o, (char*)y + o, st, nullptr, (flags & FE_ASSEMBLE) != 0,
                  brick};
    if (prec == FE_F64)
      FE_TRY(native ? fe_launch_apply_f64native(L) : fe_launch_apply_f64dw(L));
    else
      FE_TRY(fe_launch_apply_f32(L));
  }
  if (!(flags & FE_ASSEMBLE)) return FE_OK;
  // structured passes of all blocks (between bricks where the kernel fused), then inter-block
  FE_TRY(fe_launch_dss_blocks(M->blocks.data(), M->off.data(), M->nblocks, prec, y, brick[0],
                              brick[1], st));
  return prec == FE_F64 ? interblock<double>(M, (double*)y, st) : interblock<float>(M, (float*)y, st);
}
