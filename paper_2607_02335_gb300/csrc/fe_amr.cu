// fe_amr.cu -- hanging nodes through shadow cells (Appendix "Extension of DSS algorithms onto
// Non-Conforming Interfaces", Algorithm "Full DSS Operator with Hanging Node Resolution").
//
// Mesh: a coarse grid of mc^3 cells of the unit cube whose cells inside the box [lo, hi) are each
// refined into 2x2x2 fine cells.  Storage: the full coarse grid, then the fine grid of the box,
// both in layout 0.  The coarse cells inside the box are dormant and hold zeros outside the DSS;
// those touching the box boundary serve as the shadow cells that broker the exchange across the
// refinement interface.  The DSS:
//   1. clear the coarse cells of the box;
//   2. restrict-add: every coarse node J of a shadow cell receives sum_i P(i, J) r_i over the
//      copies i of its fine children that lie on the box boundary, P(i, J) = prod_d l_J_d(xi_d(i))
//      the parent's basis function J at the child node (P^T of the prolongation), one box-face
//      orientation at a time (2D tangent weights);
//   3. zero the fine copies on the box boundary (they are now represented by the shadows);
//   4. the structured DSS of the coarse grid and of the fine grid (Algorithm
//      "Dimensionally-Split Structured Summation"), shadows taking part as ordinary cells;
//   5. prolongate: every fine copy on the box boundary is set to sum_J P(i, J) u_J from its parent
//      shadow cell (an assignment, so copies shared by several children are not counted twice and
//      no vertex save-and-restore is needed);
//   6. clear the coarse cells of the box again.
// The summation kernels themselves never see the refinement.
#include <cstring>
#include <new>

#include "fe_vec.cuh"

namespace {

struct AmrGeo {
  int mc, n, p;
  int lo[3], hi[3];
  int fd[3];             // fine cells per direction of the box
  long long fine_off;    // first storage entry of the fine grid
  double P[2][FE_MAXN][FE_MAXN];  // P[h][i][j] = l_j((h + t_i) / 2): coarse basis at child nodes
};

// zero the coarse cells of the box (dormant and shadow)
template <class S>
__global__ void k_amr_clear(S* __restrict__ v, const __grid_constant__ AmrGeo g) {
  const int n3 = g.n * g.n * g.n;
  const int bx = g.hi[0] - g.lo[0], by = g.hi[1] - g.lo[1], bz = g.hi[2] - g.lo[2];
  const long long total = (long long)bx * by * bz * n3;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n3;
    const int a = (int)(e - c * n3);
    const int cx = g.lo[0] + (int)(c % bx), cy = g.lo[1] + (int)((c / bx) % by),
              cz = g.lo[2] + (int)(c / ((long long)bx * by));
    v[(((long long)cz * g.mc + cy) * g.mc + cx) * n3 + a] = S(0);
  }
}

// fine node (cell f, local a) on the box boundary?
__device__ __forceinline__ bool fine_on_bnd(const AmrGeo& g, int fx, int fy, int fz, int i, int j,
                                            int k) {
  const int X = fx * g.p + i, Y = fy * g.p + j, Z = fz * g.p + k;
  return X == 0 || X == g.fd[0] * g.p || Y == 0 || Y == g.fd[1] * g.p || Z == 0 ||
         Z == g.fd[2] * g.p;
}

// Steps 2 and 5 run per face orientation o = 2*axis + side of the box, in a fixed order; a fine
// node on the box boundary belongs to the first orientation whose face contains it, so every fine
// copy is restricted and prolongated exactly once, and a shadow node on a box edge collects the
// contributions of its faces in separate launches.  On a box face the parent's trace weights
// factor into the two tangent directions (the normal factor is 1 on the face).
__device__ __forceinline__ bool owned_by(const AmrGeo& g, int o, const int X[3]) {
  for (int o2 = 0; o2 < o; ++o2) {
    const int a2 = o2 >> 1;
    if (X[a2] == ((o2 & 1) ? g.fd[a2] * g.p : 0)) return false;
  }
  return true;
}

// step 2, orientation o: one thread per (shadow cell on that box face, node J of its face)
template <class S>
__global__ void k_amr_restrict(S* __restrict__ v, const __grid_constant__ AmrGeo g, int o) {
  const int n = g.n, n3 = n * n * n, p = g.p;
  const int axis = o >> 1, side = o & 1;
  const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
  int b[3];
  for (int a = 0; a < 3; ++a) b[a] = g.hi[a] - g.lo[a];
  const long long total = (long long)b[t1] * b[t2] * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Ja = (int)(e % n), Jb = (int)((e / n) % n);
    const long long sc = e / (n * n);
    int oc[3];  // shadow cell, box-local
    oc[axis] = side ? b[axis] - 1 : 0;
    oc[t1] = (int)(sc % b[t1]);
    oc[t2] = (int)(sc / b[t1]);
    S acc = S(0);
    for (int hb = 0; hb < 2; ++hb)
      for (int ha = 0; ha < 2; ++ha) {
        int fc[3];
        fc[axis] = 2 * oc[axis] + side;
        fc[t1] = 2 * oc[t1] + ha;
        fc[t2] = 2 * oc[t2] + hb;
        const long long fbase =
            g.fine_off + (((long long)fc[2] * g.fd[1] + fc[1]) * g.fd[0] + fc[0]) * n3;
        for (int ib = 0; ib < n; ++ib)
          for (int ia = 0; ia < n; ++ia) {
            int l[3], X[3];
            l[axis] = side ? p : 0;
            l[t1] = ia;
            l[t2] = ib;
            for (int a = 0; a < 3; ++a) X[a] = fc[a] * p + l[a];
            if (!owned_by(g, o, X)) continue;
            const double w = g.P[ha][ia][Ja] * g.P[hb][ib][Jb];
            if (w != 0.0) acc += S(w) * v[fbase + ((long long)l[2] * n + l[1]) * n + l[0]];
          }
      }
    int J[3];
    J[axis] = side ? p : 0;
    J[t1] = Ja;
    J[t2] = Jb;
    const long long cidx = (((long long)(g.lo[2] + oc[2]) * g.mc + g.lo[1] + oc[1]) * g.mc +
                            g.lo[0] + oc[0]) * n3 + ((long long)J[2] * n + J[1]) * n + J[0];
    v[cidx] += acc;
  }
}

// step 5, orientation o: one thread per (shadow cell on that box face, child on it, node)
template <class S>
__global__ void k_amr_prolong(S* __restrict__ v, const __grid_constant__ AmrGeo g, int o) {
  const int n = g.n, n3 = n * n * n, p = g.p;
  const int axis = o >> 1, side = o & 1;
  const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
  int b[3];
  for (int a = 0; a < 3; ++a) b[a] = g.hi[a] - g.lo[a];
  const long long total = (long long)b[t1] * b[t2] * 4 * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int ia = (int)(e % n), ib = (int)((e / n) % n);
    const int h = (int)((e / (n * n)) % 4), ha = h & 1, hb = h >> 1;
    const long long sc = e / (4 * n * n);
    int oc[3], fc[3], l[3], X[3];
    oc[axis] = side ? b[axis] - 1 : 0;
    oc[t1] = (int)(sc % b[t1]);
    oc[t2] = (int)(sc / b[t1]);
    fc[axis] = 2 * oc[axis] + side;
    fc[t1] = 2 * oc[t1] + ha;
    fc[t2] = 2 * oc[t2] + hb;
    l[axis] = side ? p : 0;
    l[t1] = ia;
    l[t2] = ib;
    for (int a = 0; a < 3; ++a) X[a] = fc[a] * p + l[a];
    if (!owned_by(g, o, X)) continue;
    const long long sbase = (((long long)(g.lo[2] + oc[2]) * g.mc + g.lo[1] + oc[1]) * g.mc +
                             g.lo[0] + oc[0]) * n3;
    S val = S(0);
    for (int Jb = 0; Jb < n; ++Jb)
      for (int Ja = 0; Ja < n; ++Ja) {
        const double w = g.P[ha][ia][Ja] * g.P[hb][ib][Jb];
        if (w == 0.0) continue;
        int J[3];
        J[axis] = side ? p : 0;
        J[t1] = Ja;
        J[t2] = Jb;
        val += S(w) * v[sbase + ((long long)J[2] * n + J[1]) * n + J[0]];
      }
    v[g.fine_off + (((long long)fc[2] * g.fd[1] + fc[1]) * g.fd[0] + fc[0]) * n3 +
      ((long long)l[2] * n + l[1]) * n + l[0]] = val;
  }
}

// step 3: zero the fine copies on the box boundary
template <class S>
__global__ void k_amr_fine_bnd_zero(S* __restrict__ v, const __grid_constant__ AmrGeo g) {
  const int n = g.n, n3 = n * n * n;
  const long long total = (long long)g.fd[0] * g.fd[1] * g.fd[2] * n3;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / n3;
    const int a = (int)(e - f * n3);
    const int fx = (int)(f % g.fd[0]), fy = (int)((f / g.fd[0]) % g.fd[1]),
              fz = (int)(f / ((long long)g.fd[0] * g.fd[1]));
    if (fine_on_bnd(g, fx, fy, fz, a % n, (a / n) % n, a / (n * n))) v[g.fine_off + e] = S(0);
  }
}

unsigned grid_cap(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

struct fe_amr {
  fe_amr_desc d;
  fe_mesh* coarse = nullptr;
  fe_mesh* fine = nullptr;
  AmrGeo g;
  long long len = 0, nu = 0;
};

extern "C" fe_status fe_amr_create(const fe_amr_desc* d, void* stream, fe_amr** out) {
  if (!d || !out) {
    fe_set_error("fe_amr_create: null argument");
    return FE_ERR_INVALID;
  }
  *out = nullptr;
  if (d->degree < 1 || d->degree > 7 || d->mc < 3) {
    fe_set_error("fe_amr_create: degree %d outside [1,7] or mc %d < 3", d->degree, d->mc);
    return FE_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a)
    if (!(1 <= d->lo[a] && d->lo[a] < d->hi[a] && d->hi[a] <= d->mc - 1)) {
      fe_set_error("fe_amr_create: the refined box must lie strictly inside the coarse grid");
      return FE_ERR_INVALID;
    }
  fe_amr* A = new (std::nothrow) fe_amr();
  if (!A) {
    fe_set_error("fe_amr_create: host allocation failed");
    return FE_ERR_OOM;
  }
  A->d = *d;
  const int p = d->degree, n = p + 1, mc = d->mc;
  std::memset(&A->g, 0, sizeof(A->g));
  A->g.mc = mc;
  A->g.n = n;
  A->g.p = p;
  long long fcells = 1, inner_c = 1, inner_f = 1;
  for (int a = 0; a < 3; ++a) {
    A->g.lo[a] = d->lo[a];
    A->g.hi[a] = d->hi[a];
    A->g.fd[a] = 2 * (d->hi[a] - d->lo[a]);
    fcells *= A->g.fd[a];
    inner_c *= (long long)(d->hi[a] - d->lo[a]) * p - 1;
    inner_f *= (long long)A->g.fd[a] * p - 1;
  }
  const long long n3 = (long long)n * n * n;
  A->g.fine_off = (long long)mc * mc * mc * n3;
  A->len = A->g.fine_off + fcells * n3;
  // coarse lattice nodes minus those strictly inside the box, plus the fine ones strictly inside
  A->nu = (long long)(mc * p + 1) * (mc * p + 1) * (mc * p + 1) - inner_c + inner_f;
  HostTab tab;
  fe_host_tables(p, &tab);
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i < n; ++i) {
      const double s = 0.5 * (h + tab.t[i]);
      for (int j = 0; j < n; ++j) {  // Lagrange basis j of the GLL nodes at s
        double l = 1.0;
        for (int r = 0; r < n; ++r)
          if (r != j) l *= (s - tab.t[r]) / (tab.t[j] - tab.t[r]);
        A->g.P[h][i][j] = l;
      }
    }
  fe_mesh_desc cd;
  std::memset(&cd, 0, sizeof(cd));
  cd.mx = cd.my = cd.mz = mc;
  cd.degree = p;
  cd.geom_mode = FE_GEOM_STORED;
  cd.device = d->device;
  double cc[24], fc[24];
  for (int c = 0; c < 8; ++c)
    for (int a = 0; a < 3; ++a) {
      const int bit = (c >> a) & 1;
      cc[3 * c + a] = bit;
      fc[3 * c + a] = (double)(bit ? d->hi[a] : d->lo[a]) / mc;
    }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(d->device), "cudaSetDevice");
  fe_status s = fe_mesh_create_impl(&cd, cc, stream, &A->coarse);
  if (s == FE_OK) {
    fe_mesh_desc fdsc = cd;
    fdsc.mx = A->g.fd[0];
    fdsc.my = A->g.fd[1];
    fdsc.mz = A->g.fd[2];
    s = fe_mesh_create_impl(&fdsc, fc, stream, &A->fine);
  }
  if (s != FE_OK) {
    if (A->coarse) fe_mesh_destroy(A->coarse);
    if (A->fine) fe_mesh_destroy(A->fine);
    delete A;
    return s;
  }
  *out = A;
  return FE_OK;
}

extern "C" fe_status fe_amr_destroy(fe_amr* A) {
  if (!A) return FE_OK;
  fe_mesh_destroy(A->coarse);
  fe_mesh_destroy(A->fine);
  delete A;
  return FE_OK;
}

extern "C" fe_status fe_amr_layout(const fe_amr* A, fe_layout* out) {
  if (!A || !out) {
    fe_set_error("fe_amr_layout: null argument");
    return FE_ERR_INVALID;
  }
  out->n_cells = A->coarse->ncells + A->fine->ncells;
  out->nodes_per_cell = A->coarse->n3;
  out->cellwise_len = A->len;
  out->unique_dofs = A->nu;
  out->layout_id = FE_LAYOUT_CELLS;
  return FE_OK;
}

template <class S>
static fe_status amr_dss(const fe_amr* A, S* v, cudaStream_t st) {
  const long long nbox = (long long)(A->g.hi[0] - A->g.lo[0]) * (A->g.hi[1] - A->g.lo[1]) *
                         (A->g.hi[2] - A->g.lo[2]) * A->coarse->n3;
  const long long nfine = A->fine->ncells * A->fine->n3;
  const int prec = sizeof(S) == 8 ? FE_F64 : FE_F32;
  const int n2 = A->g.n * A->g.n;
  int b[3];
  for (int a = 0; a < 3; ++a) b[a] = A->g.hi[a] - A->g.lo[a];
  auto face_items = [&](int o) {
    const int axis = o >> 1, t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
    return (long long)b[t1] * b[t2] * n2;
  };
  k_amr_clear<S><<<grid_cap(nbox, 256), 256, 0, st>>>(v, A->g);
  for (int o = 0; o < 6; ++o)
    k_amr_restrict<S><<<grid_cap(face_items(o), 128), 128, 0, st>>>(v, A->g, o);
  k_amr_fine_bnd_zero<S><<<grid_cap(nfine, 256), 256, 0, st>>>(v, A->g);
  FE_TRY(fe_launch_dss(A->coarse, prec, v, st));
  FE_TRY(fe_launch_dss(A->fine, prec, v + A->g.fine_off, st));
  for (int o = 0; o < 6; ++o)
    k_amr_prolong<S><<<grid_cap(4 * face_items(o), 128), 128, 0, st>>>(v, A->g, o);
  k_amr_clear<S><<<grid_cap(nbox, 256), 256, 0, st>>>(v, A->g);
  return fe_cuda_check(cudaGetLastError(), "hanging-node DSS launch");
}

static fe_status amr_check(const fe_amr* A, fe_prec prec, const void* a, const void* b,
                           const char* what) {
  if (!A || !a || !b) {
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

extern "C" fe_status fe_amr_dss(const fe_amr* A, fe_prec prec, const void* r, void* z,
                                void* stream) {
  FE_TRY(amr_check(A, prec, r, z, "fe_amr_dss"));
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(A->d.device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = prec == FE_F64 ? sizeof(double) : sizeof(float);
  if (r != z)
    FE_CUDA(cudaMemcpyAsync(z, r, (size_t)A->len * es, cudaMemcpyDeviceToDevice, st), "amr copy");
  return prec == FE_F64 ? amr_dss<double>(A, (double*)z, st) : amr_dss<float>(A, (float*)z, st);
}

extern "C" fe_status fe_amr_apply(const fe_amr* A, fe_op op, fe_prec prec, const void* x,
                                  void* y, unsigned flags, void* stream) {
  FE_TRY(amr_check(A, prec, x, y, "fe_amr_apply"));
  if (op != FE_LAPLACE && op != FE_MASS) {
    fe_set_error("fe_amr_apply: unknown operator %d", (int)op);
    return FE_ERR_INVALID;
  }
  if (flags & ~(FE_ASSEMBLE | FE_NATIVE_F64)) {
    fe_set_error("fe_amr_apply: unknown flags 0x%x", flags);
    return FE_ERR_INVALID;
  }
  const size_t es = prec == FE_F64 ? sizeof(double) : sizeof(float);
  const char *xb = (const char*)x, *yb = (const char*)y;
  if (xb < yb + A->len * es && yb < xb + A->len * es) {
    fe_set_error("fe_amr_apply: x and y overlap");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(A->d.device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const bool native = (flags & FE_NATIVE_F64) && prec == FE_F64;
  const fe_mesh* lv[2] = {A->coarse, A->fine};
  const size_t off[2] = {0, (size_t)A->g.fine_off * es};
  for (int l = 0; l < 2; ++l) {
    FE_TRY(fe_ensure_geometry(lv[l], prec, native));
    ApplyLaunch L{lv[l], (int)op, xb + off[l], (char*)y + off[l], st, nullptr, false};
    if (prec == FE_F64)
      FE_TRY(native ? fe_launch_apply_f64native(L) : fe_launch_apply_f64dw(L));
    else
      FE_TRY(fe_launch_apply_f32(L));
  }
  if (!(flags & FE_ASSEMBLE)) {  // dormant coarse cells carry no data
    if (prec == FE_F64)
      k_amr_clear<double><<<grid_cap(A->len, 256), 256, 0, st>>>((double*)y, A->g);
    else
      k_amr_clear<float><<<grid_cap(A->len, 256), 256, 0, st>>>((float*)y, A->g);
    return fe_cuda_check(cudaGetLastError(), "hanging-node clear launch");
  }
  return prec == FE_F64 ? amr_dss<double>(A, (double*)y, st) : amr_dss<float>(A, (float*)y, st);
}
