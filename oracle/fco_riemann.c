/*
 * fco_riemann.c -- edge solvers for the oracle (TEST INFRASTRUCTURE).
 *
 * Sec. 3 of the paper: at every edge a Riemann problem between the
 * piecewise-constant left and right states yields waves and speeds; for
 * scalar advection the single wave travels at the edge's advection speed, for
 * systems a Roe solver is used; a wave limiter removes oscillations of the
 * second-order correction.  The formulas (Roe linearisation of the 2D
 * shallow-water equations, MC limiter, transverse eigen-splitting) are those of
 * the wave-propagation method the paper cites, written out here.
 *
 * Shallow water, q = (h, hu, hv), normal direction with momentum index mn and
 * transverse index mt:
 *   u_hat = (sqrt(hL) uL + sqrt(hR) uR) / (sqrt(hL) + sqrt(hR)), v_hat alike,
 *   c_hat = sqrt(g (hL + hR) / 2),  delta = qR - qL,
 *   a1 = ((u_hat + c_hat) d0 - d[mn]) / (2 c_hat),  a2 = d[mt] - v_hat d0,
 *   a3 = (d[mn] - (u_hat - c_hat) d0) / (2 c_hat),
 *   W1 = a1 (1, u_hat - c_hat, v_hat), s1 = u_hat - c_hat,
 *   W2 = a2 (0, 0, 1),                  s2 = u_hat,
 *   W3 = a3 (1, u_hat + c_hat, v_hat), s3 = u_hat + c_hat
 * (components listed as (h, normal momentum, transverse momentum)).
 */
#include "fco_internal.h"
#include <math.h>
#include <stdlib.h>

static double minv(double a, double b) { return a < b ? a : b; }
static double maxv(double a, double b) { return a > b ? a : b; }

void fco_riemann_swe(int dir, const double *qL, const double *qR, double g, fco_edge *e)
{
    int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
    double hL = qL[0], hR = qR[0];
    double uL = qL[mn] / hL, uR = qR[mn] / hR;
    double vL = qL[mt] / hL, vR = qR[mt] / hR;
    double sL = sqrt(hL), sR = sqrt(hR);
    double uh = (sL * uL + sR * uR) / (sL + sR);
    double vh = (sL * vL + sR * vR) / (sL + sR);
    double ch = sqrt(g * (0.5 * (hL + hR)));
    double d[3] = {qR[0] - qL[0], qR[1] - qL[1], qR[2] - qL[2]};
    double a1 = ((uh + ch) * d[0] - d[mn]) / (2.0 * ch);
    double a2 = d[mt] - vh * d[0];
    double a3 = (d[mn] - (uh - ch) * d[0]) / (2.0 * ch);
    e->nw = 3;
    e->un = uh; e->ut = vh; e->c = ch;
    for (int k = 0; k < 3; ++k) { e->W[0][k] = 0.0; e->W[1][k] = 0.0; e->W[2][k] = 0.0; }
    e->W[0][0] = a1; e->W[0][mn] = a1 * (uh - ch); e->W[0][mt] = a1 * vh;
    e->W[1][mt] = a2;
    e->W[2][0] = a3; e->W[2][mn] = a3 * (uh + ch); e->W[2][mt] = a3 * vh;
    e->s[0] = uh - ch; e->s[1] = uh; e->s[2] = uh + ch;
    for (int k = 0; k < 3; ++k) {
        double am = 0.0, ap = 0.0;
        for (int p = 0; p < 3; ++p) {
            am += minv(e->s[p], 0.0) * e->W[p][k];
            ap += maxv(e->s[p], 0.0) * e->W[p][k];
        }
        e->amdq[k] = am; e->apdq[k] = ap;
    }
}

/*
 * Harten-Hyman entropy fix (LeVeque, Finite Volume Methods for Hyperbolic
 * Problems, Sec. 15.3.5).  The 1-wave is a transonic rarefaction when the
 * characteristic speed u - c is negative in the left state and positive in
 * the state between the 1- and 2-waves (qL + W1); the 3-wave when u + c is
 * negative between the 2- and 3-waves (qR - W3) and positive in the right
 * state.  Such a wave with Roe speed s and end speeds lam_l < 0 < lam_r is
 * split into a left-going part lam_l beta W and a right-going part
 * lam_r (1 - beta) W, beta = (lam_r - s) / (lam_r - lam_l), which sum to s W.
 * Every other wave contributes min(s, 0) W and max(s, 0) W as before, in the
 * same order, so an edge without a transonic wave keeps its fluctuations
 * bit for bit.
 */
void fco_entropy_fix_swe(int dir, const double *qL, const double *qR, double g, fco_edge *e)
{
    int mn = dir == 0 ? 1 : 2;
    int tr[3] = {0, 0, 0};
    double lam_l[3] = {0.0, 0.0, 0.0}, lam_r[3] = {0.0, 0.0, 0.0};
    {
        double hl = qL[0], l0 = qL[mn] / hl - sqrt(g * hl);
        double hm = hl + e->W[0][0], l1 = (qL[mn] + e->W[0][mn]) / hm - sqrt(g * hm);
        if (l0 < 0.0 && l1 > 0.0) { tr[0] = 1; lam_l[0] = l0; lam_r[0] = l1; }
    }
    {
        double hr = qR[0], l1 = qR[mn] / hr + sqrt(g * hr);
        double hm = hr - e->W[2][0], l0 = (qR[mn] - e->W[2][mn]) / hm + sqrt(g * hm);
        if (l0 < 0.0 && l1 > 0.0) { tr[2] = 1; lam_l[2] = l0; lam_r[2] = l1; }
    }
    if (!tr[0] && !tr[2]) return;
    for (int k = 0; k < 3; ++k) {
        double am = 0.0, ap = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (tr[p]) {
                double beta = (lam_r[p] - e->s[p]) / (lam_r[p] - lam_l[p]);
                am += lam_l[p] * beta * e->W[p][k];
                ap += lam_r[p] * (1.0 - beta) * e->W[p][k];
            } else {
                am += minv(e->s[p], 0.0) * e->W[p][k];
                ap += maxv(e->s[p], 0.0) * e->W[p][k];
            }
        }
        e->amdq[k] = am; e->apdq[k] = ap;
    }
}

/* scalar advection: one wave W = qR - qL moving at the edge speed */
void fco_riemann_adv(double vel, const double *qL, const double *qR, fco_edge *e)
{
    e->nw = 1;
    e->W[0][0] = qR[0] - qL[0];
    e->s[0] = vel;
    e->amdq[0] = minv(vel, 0.0) * e->W[0][0];
    e->apdq[0] = maxv(vel, 0.0) * e->W[0][0];
    e->un = vel; e->ut = 0.0; e->c = 0.0;
}

/*
 * Transverse split at an edge of direction dir: decompose the fluctuation
 * asdq on the eigenvectors of the flux Jacobian in the OTHER direction,
 * evaluated at this edge's Roe averages.  In that direction the speeds are
 * (v_hat - c, v_hat, v_hat + c) with eigenvectors r1 = (1, u_hat, v_hat - c),
 * r2 = (0, 1, 0), r3 = (1, u_hat, v_hat + c) in (h, normal, transverse)
 * components of the edge.
 */
void fco_transverse_swe(int dir, const fco_edge *e, const double *d, double *bm, double *bp)
{
    int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
    double uh = e->un, vh = e->ut, ch = e->c;
    double b1 = ((vh + ch) * d[0] - d[mt]) / (2.0 * ch);
    double b2 = d[mn] - uh * d[0];
    double b3 = (d[mt] - (vh - ch) * d[0]) / (2.0 * ch);
    double lam[3] = {vh - ch, vh, vh + ch};
    double r[3][3];
    r[0][0] = 1.0; r[0][mn] = uh; r[0][mt] = vh - ch;
    r[1][0] = 0.0; r[1][mn] = 1.0; r[1][mt] = 0.0;
    r[2][0] = 1.0; r[2][mn] = uh; r[2][mt] = vh + ch;
    double beta[3] = {b1, b2, b3};
    for (int k = 0; k < 3; ++k) {
        double m = 0.0, p = 0.0;
        for (int w = 0; w < 3; ++w) {
            m += minv(lam[w], 0.0) * beta[w] * r[w][k];
            p += maxv(lam[w], 0.0) * beta[w] * r[w][k];
        }
        bm[k] = m; bp[k] = p;
    }
}

/* MC limiter: phi(theta) = max(0, min((1 + theta)/2, 2, 2 theta)) */
double fco_mc_limiter(double theta)
{
    return maxv(0.0, minv(minv(0.5 * (1.0 + theta), 2.0), 2.0 * theta));
}

double fco_mc(double theta) { return fco_mc_limiter(theta); }

void fco_flux_swe(int dir, const double *q, double g, double *f)
{
    int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
    double h = q[0], un = q[mn] / h, ut = q[mt] / h;
    f[0] = q[mn];
    f[mn] = q[mn] * un + 0.5 * g * h * h;
    f[mt] = q[mn] * ut;
}

int fco_roe_x(const double *qL, const double *qR, double g,
              double *waves, double *s, double *amdq, double *apdq)
{
    if (!(qL[0] > 0.0) || !(qR[0] > 0.0)) return FCO_ERR_DRY;
    fco_edge e;
    fco_riemann_swe(0, qL, qR, g, &e);
    for (int p = 0; p < 3; ++p) {
        s[p] = e.s[p];
        for (int k = 0; k < 3; ++k) waves[3 * p + k] = e.W[p][k];
    }
    for (int k = 0; k < 3; ++k) { amdq[k] = e.amdq[k]; apdq[k] = e.apdq[k]; }
    return FCO_OK;
}

int fco_roe_x_efix(const double *qL, const double *qR, double g, double *amdq, double *apdq)
{
    fco_edge e;
    if (!(qL[0] > 0.0) || !(qR[0] > 0.0)) return FCO_ERR_DRY;
    fco_riemann_swe(0, qL, qR, g, &e);
    fco_entropy_fix_swe(0, qL, qR, g, &e);
    for (int k = 0; k < 3; ++k) { amdq[k] = e.amdq[k]; apdq[k] = e.apdq[k]; }
    return FCO_OK;
}

int fco_roe_transverse_x(const double *qL, const double *qR, double g,
                         const double *asdq, double *bmasdq, double *bpasdq)
{
    if (!(qL[0] > 0.0) || !(qR[0] > 0.0)) return FCO_ERR_DRY;
    fco_edge e;
    fco_riemann_swe(0, qL, qR, g, &e);
    fco_transverse_swe(0, &e, asdq, bmasdq, bpasdq);
    return FCO_OK;
}

/* ---------------------------------------------------------------------- */
/* Exact 1D shallow-water Riemann solution (for the convergence pin).      */
/* Middle depth h* solves phi(h*) = f(h*, hL) + f(h*, hR) + uR - uL = 0,    */
/* f(h, hK) = 2 (sqrt(g h) - sqrt(g hK)) for h <= hK (rarefaction),        */
/*            (h - hK) sqrt(g (h + hK) / (2 h hK)) for h > hK (shock).     */
static double fK(double h, double hK, double g)
{
    if (h <= hK) return 2.0 * (sqrt(g * h) - sqrt(g * hK));
    return (h - hK) * sqrt(g * (h + hK) / (2.0 * h * hK));
}

int fco_swe_exact(double hL, double uL, double hR, double uR, double g,
                  int n, const double *xi, double *h, double *u)
{
    if (!(hL > 0.0) || !(hR > 0.0)) return FCO_ERR_DRY;
    double lo = 1e-14, hi = 10.0 * (hL > hR ? hL : hR) + 10.0 * (fabs(uL) + fabs(uR));
    for (int it = 0; it < 200; ++it) {      /* bisection on phi(h*) */
        double mid = 0.5 * (lo + hi);
        double phi = fK(mid, hL, g) + fK(mid, hR, g) + uR - uL;
        if (phi > 0.0) hi = mid; else lo = mid;
    }
    double hs = 0.5 * (lo + hi);
    double us = 0.5 * (uL + uR) + 0.5 * (fK(hs, hR, g) - fK(hs, hL, g));
    double cL = sqrt(g * hL), cR = sqrt(g * hR), cs = sqrt(g * hs);
    for (int k = 0; k < n; ++k) {
        double x = xi[k];
        if (x <= us) {                       /* left of the contact */
            if (hs > hL) {                   /* left shock, speed from mass balance */
                double sh = (hs * us - hL * uL) / (hs - hL);
                if (x < sh) { h[k] = hL; u[k] = uL; } else { h[k] = hs; u[k] = us; }
            } else {                         /* left rarefaction fan */
                double head = uL - cL, tail = us - cs;
                if (x < head) { h[k] = hL; u[k] = uL; }
                else if (x > tail) { h[k] = hs; u[k] = us; }
                else { double c = (uL + 2.0 * cL - x) / 3.0; h[k] = c * c / g; u[k] = x + c; }
            }
        } else {                             /* right of the contact */
            if (hs > hR) {
                double sh = (hs * us - hR * uR) / (hs - hR);
                if (x > sh) { h[k] = hR; u[k] = uR; } else { h[k] = hs; u[k] = us; }
            } else {
                double head = uR + cR, tail = us + cs;
                if (x > head) { h[k] = hR; u[k] = uR; }
                else if (x < tail) { h[k] = hs; u[k] = us; }
                else { double c = (x - uR + 2.0 * cR) / 3.0; h[k] = c * c / g; u[k] = x - c; }
            }
        }
    }
    return FCO_OK;
}

/* ---------------------------------------------------------------------- */
/* 1D wave propagation with Roe waves and MC-limited corrections;          */
/* transmissive (zero-gradient) ends.  Used only by the convergence pin.   */
int fco_swe1d(int n, double dx, double dt, int nsteps, double g, double *h, double *hu)
{
    return fco_swe1d_efix(n, dx, dt, nsteps, g, 0, h, hu);
}

int fco_swe1d_efix(int n, double dx, double dt, int nsteps, double g, int efix, double *h, double *hu)
{
    const int ng = 2, N = n + 2 * ng;
    if (n < 2) return FCO_ERR_ARG;
    double *q = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *Ft = (double *)malloc(sizeof(double) * 3 * (size_t)(N + 1));
    fco_edge *e = (fco_edge *)malloc(sizeof(fco_edge) * (size_t)(N + 1));
    int rc = FCO_OK;
    const double dtdx = dt / dx;
#define Q1(k, i) q[(size_t)(k) * N + (i)]
    for (int st = 0; st < nsteps && rc == FCO_OK; ++st) {
        for (int i = 0; i < n; ++i) { Q1(0, i + ng) = h[i]; Q1(1, i + ng) = hu[i]; Q1(2, i + ng) = 0.0; }
        for (int k = 0; k < 3; ++k) {        /* zero-gradient ends */
            Q1(k, 0) = Q1(k, ng); Q1(k, 1) = Q1(k, ng);
            Q1(k, N - 1) = Q1(k, N - ng - 1); Q1(k, N - 2) = Q1(k, N - ng - 1);
        }
        for (int i = 1; i < N; ++i) {        /* edge i between cells i-1 and i */
            double qL[3] = {Q1(0, i - 1), Q1(1, i - 1), Q1(2, i - 1)};
            double qR[3] = {Q1(0, i), Q1(1, i), Q1(2, i)};
            if (!(qL[0] > 0.0) || !(qR[0] > 0.0)) { rc = FCO_ERR_DRY; break; }
            fco_riemann_swe(0, qL, qR, g, &e[i]);
            if (efix) fco_entropy_fix_swe(0, qL, qR, g, &e[i]);
        }
        if (rc) break;
        for (int i = ng; i <= N - ng; ++i) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int p = 0; p < 3; ++p) {
                int iu = e[i].s[p] >= 0.0 ? i - 1 : i + 1;
                double ww = 0.0, wu = 0.0;
                for (int k = 0; k < 3; ++k) {
                    ww += e[i].W[p][k] * e[i].W[p][k];
                    wu += e[iu].W[p][k] * e[i].W[p][k];
                }
                double phi = ww == 0.0 ? 0.0 : fco_mc_limiter(wu / ww);
                double as = fabs(e[i].s[p]);
                double c = as * (1.0 - dtdx * as);
                for (int k = 0; k < 3; ++k) acc[k] += c * (phi * e[i].W[p][k]);
            }
            for (int k = 0; k < 3; ++k) Ft[3 * i + k] = 0.5 * acc[k];
        }
        for (int i = ng; i < N - ng; ++i) {
            double X0 = (e[i].apdq[0] + e[i + 1].amdq[0]) + (Ft[3 * (i + 1)] - Ft[3 * i]);
            double X1 = (e[i].apdq[1] + e[i + 1].amdq[1]) + (Ft[3 * (i + 1) + 1] - Ft[3 * i + 1]);
            h[i - ng] = Q1(0, i) - dtdx * X0;
            hu[i - ng] = Q1(1, i) - dtdx * X1;
        }
    }
#undef Q1
    free(q); free(Ft); free(e);
    return rc;
}
