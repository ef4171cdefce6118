// Reverse mode of the reduced-sequential CTM iteration and of the bond energy
// (Sec. III, IV and the Appendix, differentiated), in FP64 on the device.
//
// Included by ctm.cu inside its internal namespace: the forward steps are the
// library's own (ein64 contractions, one-sided Jacobi SVDs), recorded on a tape
// whose entries are
//   * a pairwise contraction C = A . B ("a,b->o"): its adjoint is two more
//     pairwise contractions, dA = dC . B ("o,b->a") and dB = A . dC ("a,o->b"),
//     since every label of a contraction of the move appears in exactly two of
//     A, B, C;
//   * a truncated SVD U_k = leading k left singular vectors of M (sign-fixed):
//     the adjoint of the thin SVD M = U diag(s) V^T with the Lorentzian
//     broadening of the SVD adjoint entry point (ctm_svd_left_adjoint);
//   * a Frobenius normalisation t / ||t||: dt = (g - <g, out> out) / ||t||;
//   * a leg permutation (the rotated copies of A and B): a scatter back.
// Each CTM iteration is checkpointed: the forward pass keeps only the
// environment entering every iteration; the backward pass re-runs one
// iteration on a fresh tape and walks it backwards, from the last iteration to
// the first.

// ---------------------------------------------------------------------------
// Kernels of the reverse pass
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long rv_offset(const LegMap& m, long long idx) {
  long long off = 0;
  for (int l = m.n - 1; l >= 0; --l) {
    const long long d = m.dim[l];
    const long long q = idx / d;
    off += (idx - q * d) * m.stride[l];
    idx = q;
  }
  return off;
}

__global__ void rv_axpy_kernel(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// g_in[map(i)] += g_out[i] (map a bijection: no two i share a target)
__global__ void rv_scatter_add_kernel(double* __restrict__ g_in, const double* __restrict__ g_out,
                                      LegMap map, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    g_in[rv_offset(map, i)] += g_out[i];
}

// out = in / sqrt(nn[0])
__global__ void rv_scale_kernel(double* __restrict__ out, const double* __restrict__ in,
                                const double* __restrict__ nn, long long n) {
  const double inv = 1.0 / sqrt(nn[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i] * inv;
}

// gt += (g - dot[0] out) / sqrt(nn[0])
__global__ void rv_norm_adjoint_kernel(double* __restrict__ gt, const double* __restrict__ g,
                                       const double* __restrict__ out,
                                       const double* __restrict__ dot,
                                       const double* __restrict__ nn, long long n) {
  const double inv = 1.0 / sqrt(nn[0]), d = dot[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    gt[i] += (g[i] - d * out[i]) * inv;
}

// Thin SVD factors from a one-sided Jacobi run: column perm[j] of X (xrows long,
// orthogonal columns of norm sig) and of V (vdim long).  u_from_x: U = X / sig,
// V^T rows = V columns (Jacobi on M's columns); else U = V columns, V^T rows =
// X / sig (Jacobi on M^T's columns).  The sign of each pair is fixed so that the
// largest-magnitude entry of the U column (lowest index on ties) is positive,
// which is the convention of the library's truncated SVDs.
__global__ void rv_svd_pack_kernel(double* __restrict__ U, int urows, double* __restrict__ Vt,
                                   int vcols, double* __restrict__ s, int r,
                                   const double* __restrict__ X, int xrows,
                                   const double* __restrict__ V, int vdim,
                                   const double* __restrict__ sig, const int* __restrict__ perm,
                                   int u_from_x) {
  const int j = blockIdx.x;
  const int col = perm[j];
  const double sg = sig[col];
  const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
  const double* xc = X + (long long)col * xrows;
  const double* vc = V + (long long)col * vdim;
  __shared__ double best_v[256];
  __shared__ int best_i[256];
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < urows; i += blockDim.x) {
    const double u = u_from_x ? xc[i] * inv : vc[i];
    if (fabs(u) > bv) {
      bv = fabs(u);
      bi = i;
    }
  }
  best_v[threadIdx.x] = bv;
  best_i[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double ov = best_v[threadIdx.x + o];
      const int oi = best_i[threadIdx.x + o];
      if (ov > best_v[threadIdx.x] || (ov == best_v[threadIdx.x] && oi < best_i[threadIdx.x])) {
        best_v[threadIdx.x] = ov;
        best_i[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int im = best_i[0];
  const double um = im < urows ? (u_from_x ? xc[im] * inv : vc[im]) : 1.0;
  const double sgn = um < 0.0 ? -1.0 : 1.0;
  for (int i = threadIdx.x; i < urows; i += blockDim.x)
    U[(long long)i * r + j] = sgn * (u_from_x ? xc[i] * inv : vc[i]);
  for (int i = threadIdx.x; i < vcols; i += blockDim.x)
    Vt[(long long)j * vcols + i] = sgn * (u_from_x ? vc[i] : xc[i] * inv);
  if (threadIdx.x == 0) s[j] = sg;
}

unsigned rv_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// Tape
// ---------------------------------------------------------------------------
enum ROpKind { R_EIN = 0, R_SVD = 1, R_NORM = 2, R_PERM = 3 };

struct ROp {
  ROpKind kind;
  int a = -1, b = -1, out = -1;
  std::string spec;       // R_EIN
  LegMap map;             // R_PERM: out[i] = a[map(i)]
  int U = -1, s = -1, Vt = -1, rows = 0, cols = 0, k = 0;  // R_SVD
  int nn = -1;            // R_NORM: sum of squares of a (one element)
};

struct Tape {
  ctm_ctx* c = nullptr;
  double eps = 1e-12;
  std::vector<Tmp> store;    // owned device storage
  std::vector<int> owner;    // value -> store index
  std::vector<Ten> vals;     // value -> view (pointer + dims)
  std::vector<char> konst;   // value carries no gradient (identity projectors)
  std::vector<ROp> ops;
  std::vector<Tmp> grad;     // store index -> gradient (lazily allocated, zeroed)

  explicit Tape(ctm_ctx* ctx, double e) : c(ctx), eps(e) {}

  int own(Tmp&& t, bool is_const = false) {
    store.push_back(std::move(t));
    owner.push_back((int)store.size() - 1);
    vals.push_back(store.back().t);
    konst.push_back(is_const ? 1 : 0);
    return (int)vals.size() - 1;
  }
  int view_of(int id, std::initializer_list<int> dims) {
    Ten v = view(vals[id], dims);
    owner.push_back(owner[id]);
    vals.push_back(v);
    konst.push_back(konst[id]);
    return (int)vals.size() - 1;
  }
  const Ten& operator[](int id) const { return vals[id]; }

  // gradient buffer of value id, viewed with its dims (allocated and zeroed on first use)
  Ten grad_of(int id) {
    const int st = owner[id];
    if ((int)grad.size() < (int)store.size()) grad.resize(store.size());
    if (!grad[st].t.p) {
      const Ten& base = store[st].t;
      grad[st] = Tmp(c, base.dims, base.nd);
      ck(cudaMemsetAsync(grad[st].t.p, 0, sizeof(double) * base.size(), c->stream), "zero grad");
    }
    Ten g = vals[id];
    g.p = grad[st].t.p;
    return g;
  }
  bool has_grad(int id) const {
    const int st = owner[id];
    return st < (int)grad.size() && grad[st].t.p != nullptr;
  }
  void accumulate(int id, const Ten& x) {
    if (konst[id]) return;
    Ten g = grad_of(id);
    rv_axpy_kernel<<<rv_blocks(x.size()), 256, 0, c->stream>>>(g.p, x.p, x.size());
    ck(cudaGetLastError(), "axpy");
    ++c->launches;
  }
};

// leaf: a copy of an existing device tensor
int t_leaf(Tape& T, const Ten& src) {
  Tmp t(T.c, src.dims, src.nd);
  ck(cudaMemcpyAsync(t.t.p, src.p, sizeof(double) * src.size(), cudaMemcpyDeviceToDevice,
                     T.c->stream),
     "leaf");
  return T.own(std::move(t));
}

int t_ein(Tape& T, const char* spec, int a, int b) {
  Tmp C = ein64(T.c, spec, T[a], T[b]);
  const bool k = T.konst[a] && T.konst[b];
  const int out = T.own(std::move(C), k);
  if (!k) {
    ROp op;
    op.kind = R_EIN;
    op.a = a;
    op.b = b;
    op.out = out;
    op.spec = spec;
    T.ops.push_back(op);
  }
  return out;
}

// out[i] = a[map(i)], out shaped `dims`
int t_perm(Tape& T, int a, const LegMap& map, const int* dims, int nd) {
  Tmp o(T.c, dims, nd);
  ck(permute_f64(T.c->stream, o.t.p, T[a].p, map), "permute");
  ++T.c->launches;
  const int out = T.own(std::move(o), T.konst[a]);
  if (!T.konst[a]) {
    ROp op;
    op.kind = R_PERM;
    op.a = a;
    op.out = out;
    op.map = map;
    T.ops.push_back(op);
  }
  return out;
}

int t_normalize(Tape& T, int a) {
  const Ten& t = T[a];
  Ten flat = view(t, {(int)t.size()});
  Tmp nn = ein64(T.c, "i,i->", flat, flat);
  Tmp o(T.c, t.dims, t.nd);
  rv_scale_kernel<<<rv_blocks(t.size()), 256, 0, T.c->stream>>>(o.t.p, t.p, nn.t.p, t.size());
  ck(cudaGetLastError(), "scale");
  ++T.c->launches;
  const int out = T.own(std::move(o), T.konst[a]);
  const int nid = T.own(std::move(nn), true);
  if (!T.konst[a]) {
    ROp op;
    op.kind = R_NORM;
    op.a = a;
    op.out = out;
    op.nn = nid;
    T.ops.push_back(op);
  }
  return out;
}

// Leading k left singular vectors of value M viewed as rows x cols (exact
// one-sided Jacobi with the rotations accumulated, so that the thin factors the
// adjoint needs are at hand).  k >= rows: the identity, a constant.
int t_trunc(Tape& T, int M, int rows, int cols, int k) {
  ctm_ctx* c = T.c;
  if (k >= rows) return T.own(identity(c, rows), true);
  if (k > std::min(rows, cols)) fail(CTM_ERR_ARG, "truncation rank exceeds the matrix rank bound");
  const int r = std::min(rows, cols);
  const bool u_from_x = cols <= rows;
  const int xrows = u_from_x ? rows : cols;  // Jacobi on the r columns of M or of M^T
  Tmp X(c, {r, xrows});
  if (u_from_x) {
    LegMap m;
    push(m, cols, 1);
    push(m, rows, cols);
    ck(permute_f64(c->stream, X.t.p, T[M].p, m), "transpose");
    ++c->launches;
  } else {
    ck(cudaMemcpyAsync(X.t.p, T[M].p, sizeof(double) * (size_t)rows * cols,
                       cudaMemcpyDeviceToDevice, c->stream),
       "copy");
  }
  Tmp V(c, {r, r});
  jacobi(c, X.t.p, xrows, r, V.t.p);
  Tmp sig(c, {r});
  int* perm = (int*)dalloc(c, (r + 1) / 2 + 1);
  ck(column_norms_sorted(c->stream, X.t.p, xrows, r, sig.t.p, perm), "norms");
  Tmp U(c, {rows, r}), s(c, {r}), Vt(c, {r, cols});
  rv_svd_pack_kernel<<<r, 256, 0, c->stream>>>(U.t.p, rows, Vt.t.p, cols, s.t.p, r, X.t.p, xrows,
                                              V.t.p, r, sig.t.p, perm, u_from_x ? 1 : 0);
  ck(cudaGetLastError(), "svd pack");
  c->launches += 3;
  dfree(c, perm);
  // U_k = the leading k columns of U
  Tmp Uk(c, {rows, k});
  {
    LegMap m;
    push(m, rows, r);
    push(m, k, 1);
    ck(permute_f64(c->stream, Uk.t.p, U.t.p, m), "leading columns");
    ++c->launches;
  }
  const bool kst = T.konst[M];
  // When Jacobi runs on M's columns, a column of X whose singular value is
  // (numerically) zero normalises to noise, not to a direction orthogonal to
  // the others; the adjoint needs U to be an orthonormal basis (its columns for
  // zero values span the complement).  CholeskyQR keeps the span of every
  // leading set of columns, so it leaves the nonzero-value columns as they are
  // (to rounding) and completes the rest orthonormally.
  if (u_from_x && !kst) U = cholqr(c, U.t.p, r, 1, rows, r, 3);
  const int out = T.own(std::move(Uk), kst);
  if (!kst) {
    ROp op;
    op.kind = R_SVD;
    op.a = M;
    op.out = out;
    op.U = T.own(std::move(U), true);
    op.s = T.own(std::move(s), true);
    op.Vt = T.own(std::move(Vt), true);
    op.rows = rows;
    op.cols = cols;
    op.k = k;
    T.ops.push_back(op);
  }
  return out;
}

// ---------------------------------------------------------------------------
// Backward pass of a tape
// ---------------------------------------------------------------------------
// "a,b->o": the spec of dA = dC . B and of dB = A . dC
void adjoint_specs(const std::string& spec, std::string& sa, std::string& sb) {
  const size_t comma = spec.find(','), arrow = spec.find("->");
  const std::string a = spec.substr(0, comma), b = spec.substr(comma + 1, arrow - comma - 1);
  const std::string o = spec.substr(arrow + 2);
  sa = o + "," + b + "->" + a;
  sb = a + "," + o + "->" + b;
}

void backward(Tape& T) {
  ctm_ctx* c = T.c;
  for (int i = (int)T.ops.size() - 1; i >= 0; --i) {
    const ROp& op = T.ops[i];
    if (!T.has_grad(op.out)) continue;  // nothing downstream depends on it
    const Ten g = T.grad_of(op.out);
    switch (op.kind) {
      case R_EIN: {
        std::string sa, sb;
        adjoint_specs(op.spec, sa, sb);
        if (!T.konst[op.a]) {
          Tmp ga = ein64(c, sa.c_str(), g, T[op.b]);
          T.accumulate(op.a, ga.t);
        }
        if (!T.konst[op.b]) {
          Tmp gb = ein64(c, sb.c_str(), T[op.a], g);
          T.accumulate(op.b, gb.t);
        }
        break;
      }
      case R_PERM: {
        Ten ga = T.grad_of(op.a);
        rv_scatter_add_kernel<<<rv_blocks(g.size()), 256, 0, c->stream>>>(ga.p, g.p, op.map,
                                                                          g.size());
        ck(cudaGetLastError(), "scatter");
        ++c->launches;
        break;
      }
      case R_NORM: {
        const Ten& out = T[op.out];
        Ten gf = view(g, {(int)g.size()}), of = view(out, {(int)out.size()});
        Tmp dot = ein64(c, "i,i->", gf, of);
        Ten ga = T.grad_of(op.a);
        rv_norm_adjoint_kernel<<<rv_blocks(g.size()), 256, 0, c->stream>>>(
            ga.p, g.p, out.p, dot.t.p, T[op.nn].p, g.size());
        ck(cudaGetLastError(), "norm adjoint");
        ++c->launches;
        break;
      }
      case R_SVD: {
        Tmp gM(c, {op.rows, op.cols});
        const int rc = ctm_svd_left_adjoint(T[op.U].p, T[op.s].p, T[op.Vt].p, g.p, op.rows, op.cols,
                                            op.k, T.eps, gM.t.p, c->stream);
        if (rc != CTM_OK) fail(rc, "SVD adjoint failed");
        c->launches += 6;
        T.accumulate(op.a, gM.t);
        break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The reduced-sequential iteration on a tape (the steps of projector_seq,
// split_projector, absorb_edge_seq and column_absorb, FP64, exact SVDs)
// ---------------------------------------------------------------------------
struct TEnv {
  int id[2][4][2];  // [kind][stored slot k-1][x] -> value id
};

inline int& TE(TEnv& e, int kind, int k, int x, int r) { return e.id[kind][slot_of(k, r)][x]; }

struct TSplit {
  int v1 = -1, v2 = -1, N = -1;
};

// Sec. IV, Fig. 4a: v1 from Mt[na, D, D, nb] as (na D) x (D nb), v2 from
// N = v1^T Mt as (k1 D) x nb.
TSplit t_split(Tape& T, int Mt) {
  const Ten m = T[Mt];
  const int na = m.dims[0], D = m.dims[1], nb = m.dims[3];
  ctm_ctx* c = T.c;
  TSplit P;
  const int k1 = std::min(c->chip, na * D);
  const int U1 = t_trunc(T, Mt, na * D, D * nb, k1);
  P.v1 = T.view_of(U1, {na, D, k1});
  P.N = t_ein(T, "akc,akbz->cbz", P.v1, Mt);
  const int k2 = std::min(c->chi, k1 * D);
  const int U2 = t_trunc(T, P.N, k1 * D, nb, k2);
  P.v2 = T.view_of(U2, {k1, D, k2});
  return P;
}

// Sec. IV, Fig. 4b: the six pairwise contractions, ket then bra (the same
// contraction strings as absorb_edge_seq).
int t_absorb_edge_seq(Tape& T, int Tt, int S, const char* roles, int vp1, int vp2, int vn1,
                      int vn2) {
  char ket[6] = {'s', 0, 0, 0, 0, 0}, bra[6] = {'s', 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    switch (roles[i]) {
      case 'i': ket[i + 1] = 'k'; bra[i + 1] = 'b'; break;
      case 'o': ket[i + 1] = 'o'; bra[i + 1] = 'O'; break;
      case 'p': ket[i + 1] = 'q'; bra[i + 1] = 'Q'; break;
      case 'n': ket[i + 1] = 'n'; bra[i + 1] = 'N'; break;
      default: fail(CTM_ERR_ARG, "internal: bad role");
    }
  }
  char spec[64];
  const int X1 = t_ein(T, "AkbB,Bnc->Akbnc", Tt, vn1);
  std::snprintf(spec, sizeof spec, "Akbnc,%s->Abcsoq", ket);
  const int X2 = t_ein(T, spec, X1, S);
  const int X3 = t_ein(T, "Abcsoq,Aqe->bcsoe", X2, vp1);
  const int X4 = t_ein(T, "bcsoe,cNy->bsoeNy", X3, vn2);
  std::snprintf(spec, sizeof spec, "bsoeNy,%s->oeyOQ", bra);
  const int X5 = t_ein(T, spec, X4, S);
  return t_ein(T, "oeyOQ,eQx->xoOy", X5, vp2);
}

// Reduced-network projector of the bond below x (Sec. III-IV, Fig. 3c, Fig. 8).
TSplit t_projector_seq(Tape& T, TEnv& e, const int site[4][2], int r, int x) {
  const int S = site[r][x];
  const int C1 = TE(e, 0, 1, x, r), T1 = TE(e, 1, 1, x, r);
  const int C2 = TE(e, 0, 2, x, r), T3 = TE(e, 1, 3, x, r);
  const int T2 = TE(e, 1, 2, x, r);
  const int L = t_ein(T, "dg,akbd->gkba", C1, T1);
  const TSplit Pl = t_split(T, L);
  const int R = t_ein(T, "ez,zkbw->ekbw", C2, T3);
  const TSplit Pr = t_split(T, R);
  const int C1p = t_ein(T, "cby,cba->ya", Pl.v2, Pl.N);
  const int C2p = t_ein(T, "cby,cbw->yw", Pr.v2, Pr.N);
  const int T2p = t_absorb_edge_seq(T, T2, S, "ipon", Pl.v1, Pl.v2, Pr.v1, Pr.v2);
  const int Xm = t_ein(T, "ya,ykbz->akbz", C1p, T2p);
  const int M = t_ein(T, "akbz,zw->akbw", Xm, C2p);
  return t_split(T, M);
}

// One column absorption in frame r (Sec. II, Fig. 2a-b), reduced-sequential.
void t_column_absorb(Tape& T, TEnv& e, const int site[4][2], int r) {
  TSplit P[2];
  for (int x = 0; x < 2; ++x) P[x] = t_projector_seq(T, e, site, r, x);
  int newT[2], newC1[2], newC4[2];
  for (int x = 0; x < 2; ++x) {
    const int y = other(x);
    const int S = site[r][x];
    const TSplit& vb = P[x];
    const TSplit& vt = P[y];
    const int Xc = t_ein(T, "dg,gkbe->dkbe", TE(e, 0, 1, x, r), TE(e, 1, 2, x, r));
    const int Xc4 = t_ein(T, "lu,rkbl->rukb", TE(e, 0, 4, x, r), TE(e, 1, 4, x, r));
    newT[y] = t_absorb_edge_seq(T, TE(e, 1, 1, x, r), S, "nipo", vb.v1, vb.v2, vt.v1, vt.v2);
    const int X2 = t_ein(T, "dkc,dkbe->cbe", vt.v1, Xc);
    newC1[y] = t_ein(T, "cby,cbe->ye", vt.v2, X2);
    const int W = t_ein(T, "rukb,ukc->rcb", Xc4, vb.v1);
    newC4[y] = t_ein(T, "rcb,cby->ry", W, vb.v2);
  }
  for (int y = 0; y < 2; ++y) {
    const int tn = newT[y];
    const Ten& t = T[tn];
    // [chi_p, k, b, chi_n] as stored
    TE(e, 1, 1, y, r) = t_normalize(T, T.view_of(tn, {t.dims[0], t.dims[1], t.dims[2], t.dims[3]}));
    TE(e, 0, 1, y, r) = t_normalize(T, newC1[y]);
    TE(e, 0, 4, y, r) = t_normalize(T, newC4[y]);
  }
}

void t_iteration(Tape& T, TEnv& e, const int site[4][2]) {
  for (int dir = 0; dir < 4; ++dir) {
    t_column_absorb(T, e, site, dir);
    t_column_absorb(T, e, site, dir);
  }
}

// Sites on a tape: the leaves A, B and their rotations r = 1..3 (one quarter turn
// each: rot(A)[p, a1, a2, a3, a4] = A[p, a2, a3, a4, a1], as in ctm_init_env).
void t_sites(Tape& T, int site[4][2], int leafA, int leafB) {
  ctm_ctx* c = T.c;
  const int d = c->d, D = c->D;
  LegMap m;
  const long long D4 = (long long)D * D * D * D, D3 = (long long)D * D * D;
  push(m, d, D4);
  push(m, D, 1);
  push(m, D, D3);
  push(m, D, (long long)D * D);
  push(m, D, D);
  const int dims[5] = {d, D, D, D, D};
  site[0][0] = leafA;
  site[0][1] = leafB;
  for (int r = 1; r < 4; ++r)
    for (int x = 0; x < 2; ++x) site[r][x] = t_perm(T, site[r - 1][x], m, dims, 5);
}

// Density matrix of bond `bond` on a tape: the contraction sequence of
// expect_bond (ket and bra layers in turn).  Returns the (d^2 x d^2) value.
int t_bond_rho(Tape& T, TEnv& e, const int site[4][2], int bond) {
  ctm_ctx* c = T.c;
  const int r = (bond >= 2) ? 1 : 0;
  const int x = bond & 1, y = other(x);
  const int d = c->d, D = c->D, D2 = D * D;
  const int Sx = site[r][x], Sy = site[r][y];
  auto fused = [&](int id) {
    const Ten& t = T[id];
    return T.view_of(id, {t.dims[0], t.dims[1] * t.dims[2], t.dims[3]});
  };
  int left;
  {
    const int e1 = t_ein(T, "dg,gUe->dUe", TE(e, 0, 1, x, r), fused(TE(e, 1, 2, x, r)));
    const int e2 = t_ein(T, "dUe,mLd->mLUe", e1, fused(TE(e, 1, 1, x, r)));
    const Ten& t2 = T[e2];
    const int tv = T.view_of(e2, {t2.dims[0], D, D, D, D, t2.dims[3]});
    const int s1 = t_ein(T, "pcagh,mabcfe->pghmbfe", Sx, tv);
    const int s2 = t_ein(T, "Pfbij,pghmbfe->Pijpghme", Sx, s1);
    const int bl = t_ein(T, "kXl,lm->kXm", fused(TE(e, 1, 4, x, r)), TE(e, 0, 4, x, r));
    const Ten& b = T[bl];
    const int bv = T.view_of(bl, {b.dims[0], D, D, b.dims[2]});
    left = t_ein(T, "Pijpghme,kgim->ehjkpP", s2, bv);
  }
  int right;
  {
    const int f1 = t_ein(T, "eVz,zh->eVh", fused(TE(e, 1, 2, y, r)), TE(e, 0, 2, y, r));
    const int f2 = t_ein(T, "eVh,hWt->eVWt", f1, fused(TE(e, 1, 3, y, r)));
    const Ten& t2 = T[f2];
    const int tv = T.view_of(f2, {t2.dims[0], D, D, D, D, t2.dims[3]});
    const int s1 = t_ein(T, "qaghc,eabcft->qghebft", Sy, tv);
    const int s2 = t_ein(T, "Qbnmf,qghebft->Qnmqghet", Sy, s1);
    const int br = t_ein(T, "ti,iYk->tYk", TE(e, 0, 3, y, r), fused(TE(e, 1, 4, y, r)));
    const Ten& b = T[br];
    const int bv = T.view_of(br, {b.dims[0], D, D, b.dims[2]});
    right = t_ein(T, "Qnmqghet,thmk->egnkqQ", s2, bv);
  }
  const Ten& L = T[left];
  const Ten& R = T[right];
  const int lv = T.view_of(left, {L.dims[0], D2, L.dims[3], d, d});
  const int rv = T.view_of(right, {R.dims[0], D2, R.dims[3], d, d});
  const int rho = t_ein(T, "eRkpP,eRkqQ->pqPQ", lv, rv);
  return T.view_of(rho, {d * d, d * d});
}

// ---------------------------------------------------------------------------
// Energy and gradient with checkpointed iterations
// ---------------------------------------------------------------------------
struct EnvSnap {
  Tmp t[2][4][2];
};

void snap_copy(ctm_ctx* c, EnvSnap& s, const Ten (&src)[2][4][2]) {
  for (int kind = 0; kind < 2; ++kind)
    for (int k = 0; k < 4; ++k)
      for (int x = 0; x < 2; ++x) {
        const Ten& t = src[kind][k][x];
        s.t[kind][k][x] = Tmp(c, t.dims, t.nd);
        ck(cudaMemcpyAsync(s.t[kind][k][x].t.p, t.p, sizeof(double) * t.size(),
                           cudaMemcpyDeviceToDevice, c->stream),
           "snapshot");
      }
}

// Tape leaves for one environment snapshot and for A, B; e receives their ids.
void tape_leaves(Tape& T, const EnvSnap& s, TEnv& e, int st[4][2], int& leafA, int& leafB) {
  for (int kind = 0; kind < 2; ++kind)
    for (int k = 0; k < 4; ++k)
      for (int x = 0; x < 2; ++x) e.id[kind][k][x] = t_leaf(T, s.t[kind][k][x].t);
  Ten a, b;
  site(T.c, 0, 0, a);
  site(T.c, 0, 1, b);
  leafA = t_leaf(T, a);
  leafB = t_leaf(T, b);
  t_sites(T, st, leafA, leafB);
}

void add_into(ctm_ctx* c, Tmp& acc, const Ten& g) {
  rv_axpy_kernel<<<rv_blocks(g.size()), 256, 0, c->stream>>>(acc.t.p, g.p, g.size());
  ck(cudaGetLastError(), "axpy");
  ++c->launches;
}

// E = mean over the four bonds of <op> after `iters` reduced-sequential
// iterations from the context's current environment (held fixed); gA, gB (device
// d D^4 each) receive dE/dA and dE/dB.
double energy_grad(ctm_ctx* c, int iters, double eps, const double* op_h, Tmp& gA, Tmp& gB) {
  const int d = c->d, dd = d * d;
  std::vector<EnvSnap> snaps(iters + 1);
  snap_copy(c, snaps[0], c->env);
  for (int it = 0; it < iters; ++it) {  // forward, keeping only each iteration's input
    Tape T(c, eps);
    TEnv e;
    int site[4][2], la, lb;
    tape_leaves(T, snaps[it], e, site, la, lb);
    t_iteration(T, e, site);
    Ten out[2][4][2];
    for (int kind = 0; kind < 2; ++kind)
      for (int k = 0; k < 4; ++k)
        for (int x = 0; x < 2; ++x) out[kind][k][x] = T[e.id[kind][k][x]];
    snap_copy(c, snaps[it + 1], out);
  }
  for (Tmp* g : {&gA, &gB})
    ck(cudaMemsetAsync(g->t.p, 0, sizeof(double) * g->t.size(), c->stream), "zero");
  EnvSnap genv;
  bool have_genv = false;
  double E = 0.0;
  {
    Tape T(c, eps);
    TEnv e;
    int site[4][2], la, lb;
    tape_leaves(T, snaps[iters], e, site, la, lb);
    const TEnv e0 = e;
    std::vector<double> rho(dd * dd), seed(dd * dd);
    for (int bond = 0; bond < 4; ++bond) {
      const int rid = t_bond_rho(T, e, site, bond);
      ck(cudaMemcpyAsync(rho.data(), T[rid].p, sizeof(double) * dd * dd, cudaMemcpyDeviceToHost,
                         c->stream),
         "d2h");
      ck(cudaStreamSynchronize(c->stream), "sync");
      double num = 0.0, den = 0.0;
      for (int i = 0; i < dd; ++i) {
        den += rho[i * dd + i];
        for (int j = 0; j < dd; ++j) num += rho[i * dd + j] * op_h[j * dd + i];
      }
      if (!(std::fabs(den) > 0.0) || !std::isfinite(num / den))
        fail(CTM_ERR_NAN, "non-finite bond density matrix");
      const double Eb = num / den;
      E += 0.25 * Eb;
      // dE_b / drho = (op^T - E_b I) / tr(rho), times 1/4 for the mean
      for (int i = 0; i < dd; ++i)
        for (int j = 0; j < dd; ++j)
          seed[i * dd + j] = 0.25 * (op_h[j * dd + i] - (i == j ? Eb : 0.0)) / den;
      Tmp sd(c, {dd, dd});
      ck(cudaMemcpyAsync(sd.t.p, seed.data(), sizeof(double) * dd * dd, cudaMemcpyHostToDevice,
                         c->stream),
         "h2d");
      ck(cudaStreamSynchronize(c->stream), "sync");  // seed lives on the host stack
      T.accumulate(rid, sd.t);
    }
    backward(T);
    if (T.has_grad(la)) add_into(c, gA, T.grad_of(la));
    if (T.has_grad(lb)) add_into(c, gB, T.grad_of(lb));
    for (int kind = 0; kind < 2; ++kind)
      for (int k = 0; k < 4; ++k)
        for (int x = 0; x < 2; ++x) {
          const int id = e0.id[kind][k][x];
          const Ten& t = T[id];
          genv.t[kind][k][x] = Tmp(c, t.dims, t.nd);
          if (T.has_grad(id))
            ck(cudaMemcpyAsync(genv.t[kind][k][x].t.p, T.grad_of(id).p, sizeof(double) * t.size(),
                               cudaMemcpyDeviceToDevice, c->stream),
               "grad copy");
          else
            ck(cudaMemsetAsync(genv.t[kind][k][x].t.p, 0, sizeof(double) * t.size(), c->stream),
               "zero");
        }
    have_genv = true;
  }
  for (int it = iters - 1; it >= 0 && have_genv; --it) {  // backward, one iteration at a time
    Tape T(c, eps);
    TEnv e;
    int site[4][2], la, lb;
    tape_leaves(T, snaps[it], e, site, la, lb);
    const TEnv e0 = e;
    t_iteration(T, e, site);
    for (int kind = 0; kind < 2; ++kind)
      for (int k = 0; k < 4; ++k)
        for (int x = 0; x < 2; ++x) T.accumulate(e.id[kind][k][x], genv.t[kind][k][x].t);
    backward(T);
    if (T.has_grad(la)) add_into(c, gA, T.grad_of(la));
    if (T.has_grad(lb)) add_into(c, gB, T.grad_of(lb));
    for (int kind = 0; kind < 2; ++kind)
      for (int k = 0; k < 4; ++k)
        for (int x = 0; x < 2; ++x) {
          const int id = e0.id[kind][k][x];
          Tmp& g = genv.t[kind][k][x];
          const Ten& t = T[id];
          g = Tmp(c, t.dims, t.nd);
          if (T.has_grad(id))
            ck(cudaMemcpyAsync(g.t.p, T.grad_of(id).p, sizeof(double) * t.size(),
                               cudaMemcpyDeviceToDevice, c->stream),
               "grad copy");
          else
            ck(cudaMemsetAsync(g.t.p, 0, sizeof(double) * t.size(), c->stream), "zero");
        }
  }
  return E;
}
