/*
 * fmb_oracle.c -- plain FP64 CPU oracle of the simplified (two-parameter) Fuzzy
 * Metaballs renderer and of its analytic adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  Only the test suite, the package's smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, per pixel of one view (paper sections / equations):
 *
 *   ray      c = ((x+1/2-cx)/fx, (y+1/2-cy)/fy, 1), v_cam = c/|c|,
 *            v = R^T v_cam, o = -R^T t  (pinhole camera of Sec. 5; pose maps
 *            world to camera, x_cam = R x + t)
 *   hit      P_i = L_i L_i^T (= Sigma_i^-1), t_i = (mu_i-o)^T P_i v / (v^T P_i v)
 *            (the "linear approach" maximum-likelihood depth next to Eq. 2)
 *   distance r_i = o + v t_i - mu_i, d_i = -1/2 r_i^T P_i r_i + ln(lambda_i) (Eq. 2)
 *   density  delta_i = exp(d_i)                                          (Eq. 4)
 *   weight   w_i = exp(beta1 d_i - (beta2/eta) t_i)                      (Eq. 7)
 *   depth    D = sum_i w_i t_i / sum_i w_i                                (Eq. 3)
 *   alpha    A = 1 - exp(-sum_i delta_i)                                 (Eq. 8)
 *   normal   n_i = P_i r_i / |P_i r_i| (Eq. 17), N = sum_i w_i n_i / sum_i w_i
 *            (Eq. 3 reused for normals), n_f = N/|N|, reported in the camera
 *            frame as R n_f (Sec. 6: unit length)
 *   flow     p = o + v D; for a target pose (R_j, t_j): X = R_j p + t_j,
 *            flow = (fx X0/X2 + cx, fy X1/X2 + cy) - (x+1/2, y+1/2)  (Sec. 5:
 *            transform the point cloud with the adjacent pose, project, take the
 *            change in coordinates)
 *
 * The weights of Eq. 3 are evaluated as w_i / sum w = exp(e_i - m) / sum exp(e_j - m)
 * with e_i = beta1 d_i - (beta2/eta) t_i and m = max_i e_i.  This is an exact
 * identity of Eq. 3; it is needed in FP64 too because e_i underflows exp() for rays
 * that miss every Gaussian (d_i of a few hundred).
 *
 * Degenerate cases: |P_i r_i| = 0 gives n_i = 0; |N| = 0 gives n_f = 0.
 * lambda_i must be > 0.
 *
 * The backward pass is the analytic adjoint of exactly these steps, in the same
 * explicit-precision (P_i) form, accumulated over the given pixels: gradients of a
 * scalar loss with respect to the means, the packed Cholesky factors
 * (L00, L10, L11, L20, L21, L22), the weights lambda, the view's pose (R as a
 * free 3x3 matrix, row-major, then t) and the flow-target poses.
 *
 * Saved per-pixel values (for comparison with the CUDA path's saved planes):
 *   saved[0] = log sum_i exp(e_i)  (natural log), saved[1] = sum_i delta_i,
 *   saved[2] = |N|.
 *
 * Alpha-compositing variant (Sec. 3.3, "zero parameter model"; the *_ac entry
 * points): the weights of Eq. 3 become
 *   w_i = T_i (1 - exp(-delta_i))                                        (Eq. 9)
 *   T_i = exp(-sum_j delta_j [t_j < t_i])                                (Eq. 10)
 * evaluated literally: for every i, a sum over all j with the strict indicator
 * (so Gaussians at exactly equal depth do not attenuate each other).  Depth and
 * normal use Eq. 3 with these w_i (normalised by W = sum_i w_i; W = 0 gives
 * D = 0 and N = 0); alpha is Eq. 8 as before.  beta1, beta2 and eta are unused.
 * saved[0] = W for this variant.  Its adjoint, with wbar_i the upstream gradient
 * of w_i:
 *   wbar_i     = (Dbar (t_i - D) + Nbar . (n_i - N)) / W
 *   deltabar_k = wbar_k T_k exp(-delta_k) - sum_{i: t_k < t_i} wbar_i w_i
 *                + Abar exp(-sum delta)
 *   dbar_k = deltabar_k delta_k,  tbar_k (through Eq. 3) = Dbar w_k / W
 * (the indicator is piecewise constant in t, so it contributes nothing).
 *
 * Per-Gaussian colours (the *_c entry points): Eq. 3 with c_i in place of t_i,
 * C = sum_i w_i c_i / sum w (Sec. 3.1 blends normals and colours like depth);
 * its adjoint adds Cbar . (c_i - C) to the weight gradient of each Gaussian and
 * gives cbar_i = sum over pixels of (w_i / sum w) Cbar.
 */

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FMBO_MAX_TARGETS 2

/* ---- small 3-vector / 3x3 helpers (row-major 3x3) ---- */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void matvec(const double* M, const double* x, double* y) {
  for (int r = 0; r < 3; ++r) y[r] = M[3 * r] * x[0] + M[3 * r + 1] * x[1] + M[3 * r + 2] * x[2];
}

static void matTvec(const double* M, const double* x, double* y) {
  for (int c = 0; c < 3; ++c) y[c] = M[c] * x[0] + M[3 + c] * x[1] + M[6 + c] * x[2];
}

/* Unpack (L00, L10, L11, L20, L21, L22) into a full lower-triangular 3x3. */
static void unpack_L(const double* c, double* L) {
  L[0] = c[0]; L[1] = 0.0;  L[2] = 0.0;
  L[3] = c[1]; L[4] = c[2]; L[5] = 0.0;
  L[6] = c[3]; L[7] = c[4]; L[8] = c[5];
}

/* P = L L^T */
static void precision_from_L(const double* L, double* P) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += L[3 * r + k] * L[3 * c + k];
      P[3 * r + c] = s;
    }
}

typedef struct {
  int W, H;
  double fx, fy, cx, cy;
  double beta1, beta2, eta;
  int variant; /* 0: two-parameter weights (Eq. 7); 1: alpha compositing (Eq. 9-10) */
  const double* colors; /* K x 3 per-Gaussian colours, or NULL */
} fmbo_camera;

/* Ray of pixel p: camera-frame unit direction, world direction, origin. */
static void pixel_ray(const fmbo_camera* cam, const double* R, const double* t, long long p,
                      double* vcam, double* v, double* o, double* pix_xy) {
  int x = (int)(p % cam->W), y = (int)(p / cam->W);
  double px = x + 0.5, py = y + 0.5;
  double c[3] = {(px - cam->cx) / cam->fx, (py - cam->cy) / cam->fy, 1.0};
  double n = sqrt(dot3(c, c));
  for (int k = 0; k < 3; ++k) vcam[k] = c[k] / n;
  matTvec(R, vcam, v);
  double mt[3];
  matTvec(R, t, mt);
  for (int k = 0; k < 3; ++k) o[k] = -mt[k];
  pix_xy[0] = px;
  pix_xy[1] = py;
}

/* Per-pair quantities of Eq. 2, 4, 7 and 17 for one ray and one Gaussian. */
typedef struct {
  double P[9], m[3], Pv[3], r[3], g[3], n[3];
  double num, den, t, q, d, delta, e, gnorm;
} pair_t;

static void eval_pair(const double* mu, const double* cholp, double lam, const double* v, const double* o,
                      const fmbo_camera* cam, pair_t* s) {
  double L[9];
  unpack_L(cholp, L);
  precision_from_L(L, s->P);
  for (int k = 0; k < 3; ++k) s->m[k] = mu[k] - o[k];
  matvec(s->P, v, s->Pv);
  s->num = dot3(s->m, s->Pv);   /* (mu-o)^T P v  */
  s->den = dot3(v, s->Pv);      /* v^T P v       */
  s->t = s->num / s->den;
  for (int k = 0; k < 3; ++k) s->r[k] = v[k] * s->t - s->m[k]; /* o + v t - mu */
  matvec(s->P, s->r, s->g);
  s->q = dot3(s->r, s->g);
  s->d = -0.5 * s->q + log(lam);
  s->delta = exp(s->d);
  s->e = cam->beta1 * s->d - (cam->beta2 / cam->eta) * s->t;
  s->gnorm = sqrt(dot3(s->g, s->g));
  if (s->gnorm > 0.0)
    for (int k = 0; k < 3; ++k) s->n[k] = s->g[k] / s->gnorm;
  else
    s->n[0] = s->n[1] = s->n[2] = 0.0;
}

/* Pinhole projection of a camera-frame point. */
static void project(const fmbo_camera* cam, const double* X, double* uv) {
  uv[0] = cam->fx * X[0] / X[2] + cam->cx;
  uv[1] = cam->fy * X[1] / X[2] + cam->cy;
}

typedef struct {
  double D, A, Sdelta, lse, m, Sw, C[3];
  double N[3], Nnorm, nf[3], ncam[3];
  double p[3];
  double flow[FMBO_MAX_TARGETS][2];
} ray_out_t;

/* Forward for one ray.  ``pairs`` (size K) receives every pair's values and
 * ``what`` the normalised weights w_i / sum w, so that the backward pass can reuse
 * them; ``trans`` (alpha compositing only) the transmittances T_i. */
static void forward_ray(int K, const double* means, const double* chol, const double* weights,
                        const fmbo_camera* cam, const double* R, const double* v, const double* o,
                        const double* pix_xy, int n_targets, const double* target_poses,
                        pair_t* pairs, double* what, double* trans, ray_out_t* out) {
  double m = -INFINITY;
  for (int i = 0; i < K; ++i) {
    eval_pair(means + 3 * i, chol + 6 * i, weights[i], v, o, cam, &pairs[i]);
    if (pairs[i].e > m) m = pairs[i].e;
  }
  double Sw = 0.0, Sdelta = 0.0;
  if (cam->variant == 1) {
    /* Eq. 10 and Eq. 9, literally: T_i from every j strictly in front of i */
    for (int i = 0; i < K; ++i) {
      double S = 0.0;
      for (int j = 0; j < K; ++j)
        if (pairs[j].t < pairs[i].t) S += pairs[j].delta;
      trans[i] = exp(-S);
      what[i] = trans[i] * -expm1(-pairs[i].delta);
      Sw += what[i];
      Sdelta += pairs[i].delta;
    }
  } else {
    for (int i = 0; i < K; ++i) {
      what[i] = exp(pairs[i].e - m);
      Sw += what[i];
      Sdelta += pairs[i].delta;
    }
  }
  double D = 0.0, N[3] = {0, 0, 0};
  for (int i = 0; i < K; ++i) {
    what[i] = Sw > 0.0 ? what[i] / Sw : 0.0;
    D += what[i] * pairs[i].t;
    for (int k = 0; k < 3; ++k) N[k] += what[i] * pairs[i].n[k];
  }
  out->m = m;
  out->Sw = Sw;
  out->lse = cam->variant == 1 ? Sw : m + log(Sw);
  out->D = D;
  out->Sdelta = Sdelta;
  out->A = -expm1(-Sdelta);
  for (int k = 0; k < 3; ++k) out->N[k] = N[k];
  out->Nnorm = sqrt(dot3(N, N));
  for (int k = 0; k < 3; ++k) out->nf[k] = out->Nnorm > 0.0 ? N[k] / out->Nnorm : 0.0;
  matvec(R, out->nf, out->ncam);
  for (int k = 0; k < 3; ++k) out->p[k] = o[k] + v[k] * D;
  for (int k = 0; k < 3; ++k) out->C[k] = 0.0;
  if (cam->colors)
    for (int i = 0; i < K; ++i)
      for (int k = 0; k < 3; ++k) out->C[k] += what[i] * cam->colors[3 * i + k];
  for (int j = 0; j < n_targets; ++j) {
    const double* Rj = target_poses + 12 * j;
    const double* tj = Rj + 9;
    double X[3], uv[2];
    matvec(Rj, out->p, X);
    for (int k = 0; k < 3; ++k) X[k] += tj[k];
    project(cam, X, uv);
    out->flow[j][0] = uv[0] - pix_xy[0];
    out->flow[j][1] = uv[1] - pix_xy[1];
  }
}

/* Thread count of a call: n_threads > 0 as given, otherwise the process default
 * (recorded before any call changed it, so a single-thread call does not leave
 * later default calls on one thread). */
#ifdef _OPENMP
static int g_default_threads = 0;
static void use_threads(int n_threads) {
#pragma omp critical(fmbo_threads)
  if (g_default_threads == 0) g_default_threads = omp_get_max_threads();
  omp_set_num_threads(n_threads > 0 ? n_threads : g_default_threads);
}
#endif

static int check_args(int K, int W, int H, int n_targets, double fx, double fy, double eta) {
  if (K < 1 || W < 1 || H < 1) return 1;
  if (n_targets < 0 || n_targets > FMBO_MAX_TARGETS) return 1;
  if (!(fx > 0.0) || !(fy > 0.0) || !(eta > 0.0)) return 1;
  return 0;
}

/*
 * Forward render of ``n_pix`` pixels of one view (``pix`` = NULL: all W*H pixels in
 * row-major order).  Output layouts: depth[n], alpha[n], normal[n][3] (camera
 * frame), flow[n][n_targets][2] (pixels), saved[n][3].  Any output may be NULL.
 * Returns 0, or 1 on invalid arguments.
 */
static int forward_impl(int variant, int K, const double* means, const double* chol, const double* weights,
                        const double* colors, const double* pose, int n_targets, const double* target_poses,
                        int W, int H, double fx, double fy, double cx, double cy,
                        double beta1, double beta2, double eta,
                        long long n_pix, const long long* pix,
                        double* depth, double* alpha, double* normal, double* flow, double* saved,
                        double* color, int n_threads) {
  if (check_args(K, W, H, n_targets, fx, fy, eta)) return 1;
  fmbo_camera cam = {W, H, fx, fy, cx, cy, beta1, beta2, eta, variant, colors};
  if (!pix) n_pix = (long long)W * H;
  const double* R = pose;
  const double* t = pose + 9;
#ifdef _OPENMP
  use_threads(n_threads);
#else
  (void)n_threads;
#endif
  int failed = 0;
#pragma omp parallel
  {
    pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)K);
    double* what = (double*)malloc(sizeof(double) * (size_t)K);
    double* trans = (double*)malloc(sizeof(double) * (size_t)K);
    if (!pairs || !what || !trans) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(static)
      for (long long n = 0; n < n_pix; ++n) {
        long long p = pix ? pix[n] : n;
        double vcam[3], v[3], o[3], pxy[2];
        ray_out_t out;
        pixel_ray(&cam, R, t, p, vcam, v, o, pxy);
        forward_ray(K, means, chol, weights, &cam, R, v, o, pxy, n_targets, target_poses, pairs, what, trans,
                    &out);
        if (depth) depth[n] = out.D;
        if (alpha) alpha[n] = out.A;
        if (normal)
          for (int k = 0; k < 3; ++k) normal[3 * n + k] = out.ncam[k];
        if (flow)
          for (int j = 0; j < n_targets; ++j) {
            flow[(n * n_targets + j) * 2 + 0] = out.flow[j][0];
            flow[(n * n_targets + j) * 2 + 1] = out.flow[j][1];
          }
        if (saved) {
          saved[3 * n + 0] = out.lse;
          saved[3 * n + 1] = out.Sdelta;
          saved[3 * n + 2] = out.Nnorm;
        }
        if (color)
          for (int k = 0; k < 3; ++k) color[3 * n + k] = out.C[k];
      }
    }
    free(pairs);
    free(what);
    free(trans);
  }
  return failed ? 2 : 0;
}

int fmbo_forward(int K, const double* means, const double* chol, const double* weights,
                 const double* pose, int n_targets, const double* target_poses,
                 int W, int H, double fx, double fy, double cx, double cy,
                 double beta1, double beta2, double eta,
                 long long n_pix, const long long* pix,
                 double* depth, double* alpha, double* normal, double* flow, double* saved,
                 int n_threads) {
  return forward_impl(0, K, means, chol, weights, NULL, pose, n_targets, target_poses, W, H, fx, fy, cx, cy, beta1,
                      beta2, eta, n_pix, pix, depth, alpha, normal, flow, saved, NULL, n_threads);
}

/* Either variant with per-Gaussian colours (K x 3) and the colour plane color[n][3]. */
int fmbo_forward_c(int variant, int K, const double* means, const double* chol, const double* weights,
                   const double* colors, const double* pose, int n_targets, const double* target_poses,
                   int W, int H, double fx, double fy, double cx, double cy,
                   double beta1, double beta2, double eta,
                   long long n_pix, const long long* pix,
                   double* depth, double* alpha, double* normal, double* flow, double* saved, double* color,
                   int n_threads) {
  if (variant != 0 && variant != 1) return 1;
  return forward_impl(variant, K, means, chol, weights, colors, pose, n_targets, target_poses, W, H, fx, fy, cx,
                      cy, beta1, beta2, eta, n_pix, pix, depth, alpha, normal, flow, saved, color, n_threads);
}

/* Alpha-compositing variant (Eq. 9-10); beta1, beta2 and eta are ignored. */
int fmbo_forward_ac(int K, const double* means, const double* chol, const double* weights,
                    const double* pose, int n_targets, const double* target_poses,
                    int W, int H, double fx, double fy, double cx, double cy,
                    double beta1, double beta2, double eta,
                    long long n_pix, const long long* pix,
                    double* depth, double* alpha, double* normal, double* flow, double* saved,
                    int n_threads) {
  return forward_impl(1, K, means, chol, weights, NULL, pose, n_targets, target_poses, W, H, fx, fy, cx, cy, beta1,
                      beta2, eta, n_pix, pix, depth, alpha, normal, flow, saved, NULL, n_threads);
}

/* Accumulators of the backward pass (one set per thread). */
typedef struct {
  double *gmu, *gchol, *glam; /* K x 3, K x 6, K */
  double* gcol;                /* K x 3 (colours), or NULL */
  double gpose[12];
  double gtgt[FMBO_MAX_TARGETS][12];
} grads_t;

/*
 * Adjoint of one ray.  g_* are the upstream gradients of the ray's outputs.
 */
static void backward_ray(int K, const double* chol, const double* weights, const fmbo_camera* cam,
                         const double* R, const double* tpose, const double* vcam, const double* v,
                         const double* o, int n_targets, const double* target_poses,
                         const pair_t* pairs, const double* what, const double* trans, const ray_out_t* out,
                         double gD_in, double gA, const double* gN, const double* gF, const double* gC,
                         double* ebar, double* wbar, grads_t* acc) {
  double pbar[3] = {0, 0, 0};
  double vbar[3] = {0, 0, 0};
  double obar[3] = {0, 0, 0};
  double Rbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double tbar[3] = {0, 0, 0};

  /* flow: X = R_j p + t_j, uv = pi(X), flow = uv - pixel centre */
  for (int j = 0; j < n_targets; ++j) {
    const double* Rj = target_poses + 12 * j;
    const double* tj = Rj + 9;
    double X[3];
    matvec(Rj, out->p, X);
    for (int k = 0; k < 3; ++k) X[k] += tj[k];
    double iz = 1.0 / X[2];
    double gu = gF[2 * j + 0], gv = gF[2 * j + 1];
    /* d pi / d X = [[fx/Z, 0, -fx X/Z^2], [0, fy/Z, -fy Y/Z^2]] */
    double Xbar[3];
    Xbar[0] = gu * cam->fx * iz;
    Xbar[1] = gv * cam->fy * iz;
    Xbar[2] = -(gu * cam->fx * X[0] + gv * cam->fy * X[1]) * iz * iz;
    double pb[3];
    matTvec(Rj, Xbar, pb);
    for (int k = 0; k < 3; ++k) pbar[k] += pb[k];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) acc->gtgt[j][3 * r + c] += Xbar[r] * out->p[c];
    for (int k = 0; k < 3; ++k) acc->gtgt[j][9 + k] += Xbar[k];
  }
  /* p = o + v D */
  double gD = gD_in + dot3(v, pbar);
  for (int k = 0; k < 3; ++k) {
    obar[k] += pbar[k];
    vbar[k] += out->D * pbar[k];
  }

  /* normal: ncam = R n_f, n_f = N/|N|, N = sum_i what_i n_i */
  double Nbar[3] = {0, 0, 0};
  {
    double nfbar[3];
    matTvec(R, gN, nfbar);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Rbar[3 * r + c] += gN[r] * out->nf[c];
    if (out->Nnorm > 0.0) {
      double s = dot3(out->nf, nfbar);
      for (int k = 0; k < 3; ++k) Nbar[k] = (nfbar[k] - s * out->nf[k]) / out->Nnorm;
    }
  }

  /* alpha: A = 1 - exp(-S), S = sum delta_i */
  double Sbar = gA * exp(-out->Sdelta);

  if (cam->variant == 1) {
    /* alpha compositing: D = sum w t / W, N = sum w n / W with w_i = T_i (1 - exp(-delta_i)),
     * T_i = exp(-sum_j delta_j [t_j < t_i]); ebar[k] receives dbar_k = deltabar_k delta_k */
    const double Wt = out->Sw;
    for (int i = 0; i < K; ++i) {
      double Nd[3];
      for (int k = 0; k < 3; ++k) Nd[k] = pairs[i].n[k] - out->N[k];
      double cterm = 0.0;
      if (cam->colors && gC)
        for (int k = 0; k < 3; ++k) cterm += gC[k] * (cam->colors[3 * i + k] - out->C[k]);
      wbar[i] = Wt > 0.0 ? (gD * (pairs[i].t - out->D) + dot3(Nbar, Nd) + cterm) / Wt : 0.0;
    }
    for (int k = 0; k < K; ++k) {
      double behind = 0.0; /* sum over i strictly behind k of wbar_i w_i */
      for (int i = 0; i < K; ++i)
        if (pairs[k].t < pairs[i].t) behind += wbar[i] * what[i] * Wt;
      double deltabar = wbar[k] * trans[k] * exp(-pairs[k].delta) - behind + Sbar;
      ebar[k] = deltabar * pairs[k].delta;
    }
  } else {
    /* blend: what_i = softmax(e)_i; D = sum what t; N = sum what n.
     * what_bar_i = gD t_i + Nbar . n_i;  e_bar_i = what_i (what_bar_i - sum_j what_j what_bar_j) */
    double sbar = 0.0;
    for (int i = 0; i < K; ++i) {
      double wb = gD * pairs[i].t + dot3(Nbar, pairs[i].n);
      if (cam->colors && gC)
        for (int k = 0; k < 3; ++k) wb += gC[k] * cam->colors[3 * i + k];
      ebar[i] = wb;
      sbar += what[i] * wb;
    }
    for (int i = 0; i < K; ++i) ebar[i] = what[i] * (ebar[i] - sbar);
  }

  for (int i = 0; i < K; ++i) {
    const pair_t* s = &pairs[i];
    double dbar, tbar_i;
    if (cam->variant == 1) {
      dbar = ebar[i];
      tbar_i = gD * what[i];
    } else {
      /* e = beta1 d - (beta2/eta) t ; delta = exp(d) */
      dbar = cam->beta1 * ebar[i] + Sbar * s->delta;
      tbar_i = gD * what[i] - (cam->beta2 / cam->eta) * ebar[i];
    }
    /* n = g/|g|, nbar = what_i Nbar */
    double gbar[3] = {0, 0, 0};
    if (s->gnorm > 0.0) {
      double nb[3];
      for (int k = 0; k < 3; ++k) nb[k] = what[i] * Nbar[k];
      double sn = dot3(s->n, nb);
      for (int k = 0; k < 3; ++k) gbar[k] = (nb[k] - sn * s->n[k]) / s->gnorm;
    }
    /* d = -q/2 + ln(lambda) */
    double qbar = -0.5 * dbar;
    acc->glam[i] += dbar / weights[i];
    if (acc->gcol && gC)
      for (int k = 0; k < 3; ++k) acc->gcol[3 * i + k] += what[i] * gC[k];
    /* q = r^T P r, g = P r  (P symmetric) */
    double Pbar[9];
    double rbar[3];
    {
      double Pg[3];
      matvec(s->P, gbar, Pg);
      for (int k = 0; k < 3; ++k) rbar[k] = 2.0 * qbar * s->g[k] + Pg[k];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Pbar[3 * r + c] = qbar * s->r[r] * s->r[c] + gbar[r] * s->r[c];
    }
    /* r = v t - m */
    double mbar[3];
    for (int k = 0; k < 3; ++k) {
      vbar[k] += s->t * rbar[k];
      mbar[k] = -rbar[k];
    }
    tbar_i += dot3(v, rbar);
    /* t = num/den, num = m^T P v, den = v^T P v */
    double numbar = tbar_i / s->den;
    double denbar = -tbar_i * s->t / s->den;
    {
      double Pm[3];
      matvec(s->P, s->m, Pm);
      for (int k = 0; k < 3; ++k) {
        mbar[k] += numbar * s->Pv[k];
        vbar[k] += numbar * Pm[k] + 2.0 * denbar * s->Pv[k];
      }
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Pbar[3 * r + c] += numbar * s->m[r] * v[c] + denbar * v[r] * v[c];
    }
    /* m = mu - o */
    for (int k = 0; k < 3; ++k) {
      acc->gmu[3 * i + k] += mbar[k];
      obar[k] -= mbar[k];
    }
    /* P = L L^T  =>  Lbar = (Pbar + Pbar^T) L, lower triangle */
    {
      double L[9], S[9], G[9];
      unpack_L(chol + 6 * i, L);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) S[3 * r + c] = Pbar[3 * r + c] + Pbar[3 * c + r];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double a = 0.0;
          for (int k = 0; k < 3; ++k) a += S[3 * r + k] * L[3 * k + c];
          G[3 * r + c] = a;
        }
      acc->gchol[6 * i + 0] += G[0];
      acc->gchol[6 * i + 1] += G[3];
      acc->gchol[6 * i + 2] += G[4];
      acc->gchol[6 * i + 3] += G[6];
      acc->gchol[6 * i + 4] += G[7];
      acc->gchol[6 * i + 5] += G[8];
    }
  }

  /* v = R^T vcam, o = -R^T t */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rbar[3 * r + c] += vcam[r] * vbar[c] - tpose[r] * obar[c];
  {
    double Ro[3];
    matvec(R, obar, Ro);
    for (int k = 0; k < 3; ++k) tbar[k] -= Ro[k];
  }
  for (int k = 0; k < 9; ++k) acc->gpose[k] += Rbar[k];
  for (int k = 0; k < 3; ++k) acc->gpose[9 + k] += tbar[k];
}

/*
 * Gradients of sum_n [g_depth[n] D_n + g_alpha[n] A_n + g_normal[n] . ncam_n +
 * sum_j g_flow[n][j] . flow_nj] with respect to the scene and the poses, over the
 * given pixels.  Outputs are overwritten: grad_means[K][3], grad_chol[K][6],
 * grad_weights[K], grad_pose[12] (R row-major, then t), grad_target_poses
 * [n_targets][12].  Any upstream array may be NULL (treated as zero).  The result
 * is deterministic for a fixed ``n_threads``.  Returns 0, 1 on invalid arguments,
 * 2 on allocation failure.
 */
static int backward_impl(int variant, int K, const double* means, const double* chol, const double* weights,
                         const double* colors, const double* pose, int n_targets, const double* target_poses,
                         int W, int H, double fx, double fy, double cx, double cy,
                         double beta1, double beta2, double eta,
                         long long n_pix, const long long* pix,
                         const double* g_depth, const double* g_alpha, const double* g_normal,
                         const double* g_flow, const double* g_color, double* grad_means, double* grad_chol,
                         double* grad_weights, double* grad_colors, double* grad_pose, double* grad_target_poses,
                         int n_threads) {
  if (check_args(K, W, H, n_targets, fx, fy, eta)) return 1;
  fmbo_camera cam = {W, H, fx, fy, cx, cy, beta1, beta2, eta, variant, colors};
  if (!pix) n_pix = (long long)W * H;
  const double* R = pose;
  const double* t = pose + 9;
  int nt = 1;
#ifdef _OPENMP
  use_threads(n_threads);
  nt = omp_get_max_threads();
#else
  (void)n_threads;
#endif
  grads_t* accs = (grads_t*)calloc((size_t)nt, sizeof(grads_t));
  if (!accs) return 2;
  int failed = 0;
  for (int a = 0; a < nt; ++a) {
    accs[a].gmu = (double*)calloc((size_t)K * 3, sizeof(double));
    accs[a].gchol = (double*)calloc((size_t)K * 6, sizeof(double));
    accs[a].glam = (double*)calloc((size_t)K, sizeof(double));
    accs[a].gcol = (colors && grad_colors) ? (double*)calloc((size_t)K * 3, sizeof(double)) : NULL;
    if (!accs[a].gmu || !accs[a].gchol || !accs[a].glam || ((colors && grad_colors) && !accs[a].gcol)) failed = 1;
  }
  if (!failed) {
#pragma omp parallel num_threads(nt)
    {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      grads_t* acc = &accs[tid];
      pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)K);
      double* what = (double*)malloc(sizeof(double) * (size_t)K);
      double* ebar = (double*)malloc(sizeof(double) * (size_t)K);
      double* trans = (double*)malloc(sizeof(double) * (size_t)K);
      double* wbar = (double*)malloc(sizeof(double) * (size_t)K);
      if (!pairs || !what || !ebar || !trans || !wbar) {
#pragma omp atomic write
        failed = 1;
      } else {
#pragma omp for schedule(static)
        for (long long n = 0; n < n_pix; ++n) {
          long long p = pix ? pix[n] : n;
          double vcam[3], v[3], o[3], pxy[2];
          ray_out_t out;
          pixel_ray(&cam, R, t, p, vcam, v, o, pxy);
          forward_ray(K, means, chol, weights, &cam, R, v, o, pxy, n_targets, target_poses, pairs, what, trans,
                      &out);
          double gD = g_depth ? g_depth[n] : 0.0;
          double gA = g_alpha ? g_alpha[n] : 0.0;
          double gN[3] = {0, 0, 0};
          double gF[2 * FMBO_MAX_TARGETS] = {0, 0, 0, 0};
          if (g_normal)
            for (int k = 0; k < 3; ++k) gN[k] = g_normal[3 * n + k];
          if (g_flow)
            for (int j = 0; j < n_targets; ++j) {
              gF[2 * j] = g_flow[(n * n_targets + j) * 2];
              gF[2 * j + 1] = g_flow[(n * n_targets + j) * 2 + 1];
            }
          double gC[3] = {0, 0, 0};
          if (g_color)
            for (int k = 0; k < 3; ++k) gC[k] = g_color[3 * n + k];
          backward_ray(K, chol, weights, &cam, R, t, vcam, v, o, n_targets, target_poses, pairs, what, trans,
                       &out, gD, gA, gN, gF, g_color ? gC : NULL, ebar, wbar, acc);
        }
      }
      free(pairs);
      free(what);
      free(ebar);
      free(trans);
      free(wbar);
    }
  }
  if (!failed) {
    /* fixed-order reduction over the thread accumulators */
    for (int i = 0; i < 3 * K; ++i) grad_means[i] = 0.0;
    for (int i = 0; i < 6 * K; ++i) grad_chol[i] = 0.0;
    for (int i = 0; i < K; ++i) grad_weights[i] = 0.0;
    if (colors && grad_colors)
      for (int i = 0; i < 3 * K; ++i) grad_colors[i] = 0.0;
    if (grad_pose)
      for (int i = 0; i < 12; ++i) grad_pose[i] = 0.0;
    if (grad_target_poses)
      for (int i = 0; i < 12 * n_targets; ++i) grad_target_poses[i] = 0.0;
    for (int a = 0; a < nt; ++a) {
      for (int i = 0; i < 3 * K; ++i) grad_means[i] += accs[a].gmu[i];
      for (int i = 0; i < 6 * K; ++i) grad_chol[i] += accs[a].gchol[i];
      for (int i = 0; i < K; ++i) grad_weights[i] += accs[a].glam[i];
      if (accs[a].gcol)
        for (int i = 0; i < 3 * K; ++i) grad_colors[i] += accs[a].gcol[i];
      if (grad_pose)
        for (int i = 0; i < 12; ++i) grad_pose[i] += accs[a].gpose[i];
      if (grad_target_poses)
        for (int j = 0; j < n_targets; ++j)
          for (int i = 0; i < 12; ++i) grad_target_poses[12 * j + i] += accs[a].gtgt[j][i];
    }
  }
  for (int a = 0; a < nt; ++a) {
    free(accs[a].gmu);
    free(accs[a].gchol);
    free(accs[a].glam);
    free(accs[a].gcol);
  }
  free(accs);
  return failed ? 2 : 0;
}

int fmbo_backward(int K, const double* means, const double* chol, const double* weights,
                  const double* pose, int n_targets, const double* target_poses,
                  int W, int H, double fx, double fy, double cx, double cy,
                  double beta1, double beta2, double eta,
                  long long n_pix, const long long* pix,
                  const double* g_depth, const double* g_alpha, const double* g_normal, const double* g_flow,
                  double* grad_means, double* grad_chol, double* grad_weights,
                  double* grad_pose, double* grad_target_poses, int n_threads) {
  return backward_impl(0, K, means, chol, weights, NULL, pose, n_targets, target_poses, W, H, fx, fy, cx, cy,
                       beta1, beta2, eta, n_pix, pix, g_depth, g_alpha, g_normal, g_flow, NULL, grad_means,
                       grad_chol, grad_weights, NULL, grad_pose, grad_target_poses, n_threads);
}

/* Either variant with per-Gaussian colours: g_color[n][3] upstream, grad_colors [K][3]. */
int fmbo_backward_c(int variant, int K, const double* means, const double* chol, const double* weights,
                    const double* colors, const double* pose, int n_targets, const double* target_poses,
                    int W, int H, double fx, double fy, double cx, double cy,
                    double beta1, double beta2, double eta,
                    long long n_pix, const long long* pix,
                    const double* g_depth, const double* g_alpha, const double* g_normal, const double* g_flow,
                    const double* g_color, double* grad_means, double* grad_chol, double* grad_weights,
                    double* grad_colors, double* grad_pose, double* grad_target_poses, int n_threads) {
  if (variant != 0 && variant != 1) return 1;
  return backward_impl(variant, K, means, chol, weights, colors, pose, n_targets, target_poses, W, H, fx, fy, cx,
                       cy, beta1, beta2, eta, n_pix, pix, g_depth, g_alpha, g_normal, g_flow, g_color, grad_means,
                       grad_chol, grad_weights, grad_colors, grad_pose, grad_target_poses, n_threads);
}

/* Adjoint of the alpha-compositing variant (Eq. 9-10); beta1, beta2, eta ignored. */
int fmbo_backward_ac(int K, const double* means, const double* chol, const double* weights,
                     const double* pose, int n_targets, const double* target_poses,
                     int W, int H, double fx, double fy, double cx, double cy,
                     double beta1, double beta2, double eta,
                     long long n_pix, const long long* pix,
                     const double* g_depth, const double* g_alpha, const double* g_normal, const double* g_flow,
                     double* grad_means, double* grad_chol, double* grad_weights,
                     double* grad_pose, double* grad_target_poses, int n_threads) {
  return backward_impl(1, K, means, chol, weights, NULL, pose, n_targets, target_poses, W, H, fx, fy, cx, cy,
                       beta1, beta2, eta, n_pix, pix, g_depth, g_alpha, g_normal, g_flow, NULL, grad_means,
                       grad_chol, grad_weights, NULL, grad_pose, grad_target_poses, n_threads);
}

/*
 * Oriented point export of Sec. 6, for ``n_pix`` pixels of one view (``pix`` = NULL:
 * all), with the variant's weights (0: Eq. 7, 1: Eq. 9-10).  Per pixel, world frame:
 *   points[n][3]        p = o + v D, the rendered point (D from Eq. 3)
 *   normal_tf[n][3]     Eq. 17's per-Gaussian normal evaluated at the rendered depth
 *                       instead of the hit depth, n_i = P_i (o + v D - mu_i) / |.|,
 *                       blended by Eq. 3, renormalised, and turned to face the camera
 *                       (negated when n . v > 0); 0 where the blend vanishes
 *   normal_screen[n][3] Eq. 16: (p - p_x) x (p - p_y) / |.| with p_x, p_y the rendered
 *                       points of the right and lower neighbour pixels (the left /
 *                       upper one on the last column / row), turned to face the camera;
 *                       0 without a neighbour or for a zero cross product
 *   quality[n]          max_i w_i / sum_j w_j, the direct-intersection quality Sec. 6
 *                       thresholds (typically at 0.9)
 * Any output may be NULL.  Returns 0, 1 on invalid arguments, 2 on allocation failure.
 */
static void face_camera(double* n, const double* v) {
  if (dot3(n, v) > 0.0)
    for (int k = 0; k < 3; ++k) n[k] = -n[k];
}

int fmbo_points(int variant, int K, const double* means, const double* chol, const double* weights,
                const double* pose, int W, int H, double fx, double fy, double cx, double cy,
                double beta1, double beta2, double eta, long long n_pix, const long long* pix,
                double* points, double* normal_tf, double* normal_screen, double* quality, int n_threads) {
  if (check_args(K, W, H, 0, fx, fy, eta) || (variant != 0 && variant != 1)) return 1;
  fmbo_camera cam = {W, H, fx, fy, cx, cy, beta1, beta2, eta, variant, NULL};
  if (!pix) n_pix = (long long)W * H;
  const double* R = pose;
  const double* t = pose + 9;
#ifdef _OPENMP
  use_threads(n_threads);
#else
  (void)n_threads;
#endif
  int failed = 0;
#pragma omp parallel
  {
    pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)K);
    double* what = (double*)malloc(sizeof(double) * (size_t)K);
    double* trans = (double*)malloc(sizeof(double) * (size_t)K);
    if (!pairs || !what || !trans) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(static)
      for (long long n = 0; n < n_pix; ++n) {
        long long p = pix ? pix[n] : n;
        double vcam[3], v[3], o[3], pxy[2];
        ray_out_t out;
        pixel_ray(&cam, R, t, p, vcam, v, o, pxy);
        forward_ray(K, means, chol, weights, &cam, R, v, o, pxy, 0, NULL, pairs, what, trans, &out);
        if (points)
          for (int k = 0; k < 3; ++k) points[3 * n + k] = out.p[k];
        if (quality) {
          double q = 0.0;
          for (int i = 0; i < K; ++i)
            if (what[i] > q) q = what[i];
          quality[n] = q;
        }
        if (normal_tf) {
          double N[3] = {0, 0, 0};
          for (int i = 0; i < K; ++i) {
            double L[9], P[9], r[3], g[3];
            unpack_L(chol + 6 * i, L);
            precision_from_L(L, P);
            for (int k = 0; k < 3; ++k) r[k] = out.p[k] - means[3 * i + k];
            matvec(P, r, g);
            double gn = sqrt(dot3(g, g));
            if (gn > 0.0)
              for (int k = 0; k < 3; ++k) N[k] += what[i] * g[k] / gn;
          }
          double Nn = sqrt(dot3(N, N));
          for (int k = 0; k < 3; ++k) normal_tf[3 * n + k] = Nn > 0.0 ? N[k] / Nn : 0.0;
          face_camera(normal_tf + 3 * n, v);
        }
        if (normal_screen) {
          int x = (int)(p % W), y = (int)(p / W);
          double* ns = normal_screen + 3 * n;
          ns[0] = ns[1] = ns[2] = 0.0;
          if (W > 1 && H > 1) {
            long long nb[2] = {(long long)y * W + (x + 1 < W ? x + 1 : x - 1),
                               (long long)(y + 1 < H ? y + 1 : y - 1) * W + x};
            double d[2][3];
            for (int j = 0; j < 2; ++j) {
              double vc2[3], v2[3], o2[3], pxy2[2];
              ray_out_t o_nb;
              pixel_ray(&cam, R, t, nb[j], vc2, v2, o2, pxy2);
              forward_ray(K, means, chol, weights, &cam, R, v2, o2, pxy2, 0, NULL, pairs, what, trans, &o_nb);
              for (int k = 0; k < 3; ++k) d[j][k] = out.p[k] - o_nb.p[k];
            }
            double c[3] = {d[0][1] * d[1][2] - d[0][2] * d[1][1], d[0][2] * d[1][0] - d[0][0] * d[1][2],
                           d[0][0] * d[1][1] - d[0][1] * d[1][0]};
            double cn = sqrt(dot3(c, c));
            if (cn > 0.0)
              for (int k = 0; k < 3; ++k) ns[k] = c[k] / cn;
            face_camera(ns, v);
          }
        }
      }
    }
    free(pairs);
    free(what);
    free(trans);
  }
  return failed ? 2 : 0;
}

/*
 * Loss attribution of Sec. 8 (the input of the splitting criterion, Eq. 19): for
 * every Gaussian i, attribution[i] = sum over the given pixels j of
 * ray_loss[j] * w_ij / sum_k w_kj, with the variant's weights (0: Eq. 7,
 * 1: Eq. 9-10).  The paper's average over a batch of M rays is this sum / M.
 * Deterministic (serial over pixels).  Returns 0, or 1 on invalid arguments, 2 on
 * allocation failure.
 */
int fmbo_attribution(int variant, int K, const double* means, const double* chol, const double* weights,
                     const double* pose, int W, int H, double fx, double fy, double cx, double cy,
                     double beta1, double beta2, double eta, long long n_pix, const long long* pix,
                     const double* ray_loss, double* attribution) {
  if (check_args(K, W, H, 0, fx, fy, eta) || (variant != 0 && variant != 1) || !ray_loss || !attribution)
    return 1;
  fmbo_camera cam = {W, H, fx, fy, cx, cy, beta1, beta2, eta, variant, NULL};
  if (!pix) n_pix = (long long)W * H;
  pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (size_t)K);
  double* what = (double*)malloc(sizeof(double) * (size_t)K);
  double* trans = (double*)malloc(sizeof(double) * (size_t)K);
  int failed = !pairs || !what || !trans;
  if (!failed) {
    for (int i = 0; i < K; ++i) attribution[i] = 0.0;
    for (long long n = 0; n < n_pix; ++n) {
      long long p = pix ? pix[n] : n;
      double vcam[3], v[3], o[3], pxy[2];
      ray_out_t out;
      pixel_ray(&cam, pose, pose + 9, p, vcam, v, o, pxy);
      forward_ray(K, means, chol, weights, &cam, pose, v, o, pxy, 0, NULL, pairs, what, trans, &out);
      for (int i = 0; i < K; ++i) attribution[i] += ray_loss[n] * what[i];
    }
  }
  free(pairs);
  free(what);
  free(trans);
  return failed ? 2 : 0;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int fmbo_max_threads(void) {
#ifdef _OPENMP
  use_threads(0);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
