// Small dense FP64 algebra of GCRO-DR (Algorithm 3), run by one warp on the GPU:
//  * Givens update of the Hessenberg least-squares problem after each Arnoldi step;
//  * end of a cycle: least squares solution, residual/solution update coefficients, the
//    harmonic Ritz eigenproblem (first cycle: H_m + h^2 H_m^-T e_m e_m^T; later cycles:
//    the pencil G^T G z = theta G^T W^T V z, reduced to the standard problem of
//    R_G^-1 Q_G^T (W^T V) with G = Q_G R_G), eigenvector selection and QR(G P_k);
//  * Cholesky of the Gram matrix for the QR of A~ Y~ (carry to the next system).
// Eigenvalues: Householder reduction to Hessenberg form (FP64) and Francis double-shift QR on
// an FP32 copy (the eigenvalues only steer the selection and the shifts); eigenvectors of the
// selected eigenvalues by FP64 inverse iteration on the Hessenberg matrix, one warp per
// eigenvalue. All loops over rows/columns are split across the 32 lanes of a warp; scalar parts
// are computed redundantly by every lane from shared memory.
#include "gir_internal.cuh"
#include "k_small.cuh"

namespace gir {

#define LANE (threadIdx.x & 31)
#define WSYNC() __syncwarp()

__device__ __forceinline__ double sgn(double a, double b) { return b >= 0.0 ? fabs(a) : -fabs(a); }

// ------------------------------------------------------------------ Givens step
// One thread: the Givens update of column j (also called from the persistent batch kernel).
static __device__ void givens_step_dev(SmallState* st) {
    const int j = st->j, kc = st->kc;
    // column j of B (first kc coefficients) and H (next j+1) from both CGS passes
    for (int i = 0; i < kc; ++i) st->B[i + j * SM_KMAX] = st->s1[i] + st->s2[i];
    double col[SM_MMAX + 1];
    for (int i = 0; i <= j; ++i) {
        double v = st->s1[kc + i] + st->s2[kc + i];
        st->H[i + j * SM_LDH] = v;
        col[i] = v;
    }
    const double h = st->hnorm;
    st->H[j + 1 + j * SM_LDH] = h;
    col[j + 1] = h;
    for (int i = 0; i < j; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = st->cs[i] * a + st->sn[i] * b;
        col[i + 1] = -st->sn[i] * a + st->cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double rho = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (rho != 0.0) { c = a / rho; s = b / rho; }
    st->cs[j] = c;
    st->sn[j] = s;
    col[j] = rho;
    col[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) st->Hr[i + j * SM_LDH] = col[i];
    double gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->est = fabs(st->g[j + 1]);
    st->breakdown = (h == 0.0);
    st->hinv = (h != 0.0) ? 1.0 / h : 0.0;
    st->converged = (st->est <= st->tol) || (h == 0.0);
    if (!(st->est == st->est) || !(fabs(h) <= 1.7976931348623157e308)) st->status |= DEV_NONFINITE;
    st->j = j + 1;
}

// ------------------------------------------------------------------ warp helpers
static __device__ double wsum(double v) { return warp_sum(v); }

// Householder QR of the rows x cols column-major matrix X (ld) in place; R in the upper
// triangle, reflector vectors below (v[0] implicit 1), tau[] the coefficients. Positive R_ii
// is NOT enforced here.
static __device__ void house_qr(double* X, int ld, int rows, int cols, double* tau) {
    const int lane = LANE;
    for (int k = 0; k < cols && k < rows; ++k) {
        // norm of X[k:rows, k]
        double ss = 0.0;
        for (int i = k + 1 + lane; i < rows; i += 32) ss += X[i + k * ld] * X[i + k * ld];
        ss = wsum(ss);
        double alpha = X[k + k * ld];
        double nrm = sqrt(alpha * alpha + ss);
        double t = 0.0, beta = alpha;
        if (ss != 0.0 || alpha < 0.0) {
            beta = (alpha <= 0.0) ? nrm : -nrm;
            t = (beta - alpha) / beta;
            double sc = 1.0 / (alpha - beta);
            WSYNC();
            for (int i = k + 1 + lane; i < rows; i += 32) X[i + k * ld] *= sc;
        }
        WSYNC();
        if (lane == 0) { X[k + k * ld] = beta; tau[k] = t; }
        WSYNC();
        if (t != 0.0) {
            // apply (I - t v v^T) to columns k+1..cols-1, v = [1; X[k+1:, k]]
            for (int c = k + 1 + lane; c < cols; c += 32) {
                double d = X[k + c * ld];
                for (int i = k + 1; i < rows; ++i) d += X[i + k * ld] * X[i + c * ld];
                d *= t;
                X[k + c * ld] -= d;
                for (int i = k + 1; i < rows; ++i) X[i + c * ld] -= d * X[i + k * ld];
            }
        }
        WSYNC();
    }
}

// Apply Q^T (from house_qr of X) to the rows x q matrix Y (ld ldy), in place.
static __device__ void house_apply_qt(const double* X, int ld, int rows, int cols, const double* tau, double* Y, int ldy,
                               int q) {
    const int lane = LANE;
    for (int k = 0; k < cols && k < rows; ++k) {
        double t = tau[k];
        if (t == 0.0) continue;
        for (int c = lane; c < q; c += 32) {
            double d = Y[k + c * ldy];
            for (int i = k + 1; i < rows; ++i) d += X[i + k * ld] * Y[i + c * ldy];
            d *= t;
            Y[k + c * ldy] -= d;
            for (int i = k + 1; i < rows; ++i) Y[i + c * ldy] -= d * X[i + k * ld];
        }
        WSYNC();
    }
}

// Form the first q columns of Q (rows x q, ld ldq) from house_qr reflectors.
static __device__ void house_form_q(const double* X, int ld, int rows, int cols, const double* tau, double* Q, int ldq,
                             int q) {
    const int lane = LANE;
    for (int c = lane; c < q; c += 32)
        for (int i = 0; i < rows; ++i) Q[i + c * ldq] = (i == c) ? 1.0 : 0.0;
    WSYNC();
    for (int k = min(cols, rows) - 1; k >= 0; --k) {
        double t = tau[k];
        if (t == 0.0) continue;
        for (int c = lane; c < q; c += 32) {
            double d = Q[k + c * ldq];
            for (int i = k + 1; i < rows; ++i) d += X[i + k * ld] * Q[i + c * ldq];
            d *= t;
            Q[k + c * ldq] -= d;
            for (int i = k + 1; i < rows; ++i) Q[i + c * ldq] -= d * X[i + k * ld];
        }
        WSYNC();
    }
}

// Reduce M (d x d, ld) to upper Hessenberg form in place; Qh (global, ld d) accumulates the
// orthogonal similarity: M_orig = Qh Hm Qh^T. v scratch of length d.
static __device__ void hess_reduce(double* M, int ld, int d, double* Qh, double* v) {
    const int lane = LANE;
    for (int e = lane; e < d * d; e += 32) Qh[e] = ((e % d) == (e / d)) ? 1.0 : 0.0;
    WSYNC();
    for (int k = 0; k + 2 < d; ++k) {
        double ss = 0.0;
        for (int i = k + 2 + lane; i < d; i += 32) ss += M[i + k * ld] * M[i + k * ld];
        ss = wsum(ss);
        if (ss == 0.0) continue;
        double alpha = M[k + 1 + k * ld];
        double nrm = sqrt(alpha * alpha + ss);
        double beta = (alpha <= 0.0) ? nrm : -nrm;
        double t = (beta - alpha) / beta;
        double sc = 1.0 / (alpha - beta);
        // v = [0..0, 1, M[k+2:, k] * sc]
        for (int i = lane; i < d; i += 32) v[i] = (i < k + 1) ? 0.0 : (i == k + 1 ? 1.0 : M[i + k * ld] * sc);
        WSYNC();
        // left: M = (I - t v v^T) M on columns k..d-1
        for (int c = k + lane; c < d; c += 32) {
            double s = 0.0;
            for (int i = k + 1; i < d; ++i) s += v[i] * M[i + c * ld];
            s *= t;
            for (int i = k + 1; i < d; ++i) M[i + c * ld] -= s * v[i];
        }
        WSYNC();
        // right: M = M (I - t v v^T) on rows 0..d-1
        for (int r = lane; r < d; r += 32) {
            double s = 0.0;
            for (int i = k + 1; i < d; ++i) s += M[r + i * ld] * v[i];
            s *= t;
            for (int i = k + 1; i < d; ++i) M[r + i * ld] -= s * v[i];
            double q = 0.0;
            for (int i = k + 1; i < d; ++i) q += Qh[r + i * d] * v[i];
            q *= t;
            for (int i = k + 1; i < d; ++i) Qh[r + i * d] -= q * v[i];
        }
        WSYNC();
        for (int i = k + 2 + lane; i < d; i += 32) M[i + k * ld] = 0.0;
        WSYNC();
    }
}

// ------------------------------------------------------------------ Hessenberg QR eigenvalues
// Eigenvalues of an upper Hessenberg matrix by the implicitly double-shifted QR iteration
// (Francis; Golub & Van Loan, "Matrix Computations", Sec. 7.5). Written from the algorithm:
//  * the active window [lo, hi] is the unreduced block at the bottom of the part not yet
//    resolved; a subdiagonal entry is negligible (set to zero, splitting the matrix) when it is
//    at most the working precision's epsilon times the sum of its two diagonal neighbours;
//  * a 1 x 1 window gives a real eigenvalue, a 2 x 2 window a real pair or a conjugate pair
//    (closed form, below);
//  * otherwise one double-shift step: the shifts are the eigenvalues of the trailing 2 x 2 of
//    the window, entered through their sum s and product t; the first column of
//    (H - a I)(H - b I) = H^2 - s H + t I has three nonzeros, a 3-element Householder reflector
//    maps it to e_1, and further 3-element reflectors chase the bulge down the subdiagonal
//    (a 2-element one at the end). Only eigenvalues are wanted, so each reflector is applied
//    to the window only;
//  * a window that has gone 10 steps without a split takes one step with an ad hoc real
//    double shift (the last diagonal entry moved by 1.5 times the size of the last two
//    subdiagonal entries) to break a possible cycle.
// One warp: the row and column updates of each reflector are spread over the lanes; the
// reflector and the scalars are computed by every lane from shared memory.
// T = float (the default, GB300 issues dependent FP32 chains far faster than FP64 ones) or
// double. Pairs are stored as (re, +im), (re, -im). Returns 0, or 1 if the step budget
// (30 per eigenvalue) ran out; the unresolved window then reports its diagonal entries.

template <typename T> struct EpsOf;
template <> struct EpsOf<float> { static __device__ float v() { return 5.9604645e-08f; } };
template <> struct EpsOf<double> { static __device__ double v() { return 1.1102230246251565e-16; } };

// Eigenvalues of [[a, b], [c, e]] into (r1, i1), (r2, i2): with m = (a + e) / 2, h = (a - e) / 2
// and D = h^2 + b c they are m +- sqrt(D). For D >= 0 the root away from m is formed by
// addition without cancellation and the other one from the product of the two, det = a e - b c.
template <typename T>
static __device__ void eig2x2(T a, T b, T c, T e, T& r1, T& i1, T& r2, T& i2) {
    const T m = T(0.5) * (a + e), h = T(0.5) * (a - e);
    const T D = h * h + b * c;
    if (D >= T(0)) {
        const T root = sqrt(D);
        const T far = (m >= T(0)) ? m + root : m - root;
        const T det = a * e - b * c;
        r1 = far;
        r2 = (far != T(0)) ? det / far : m;
        i1 = i2 = T(0);
    } else {
        const T root = sqrt(-D);
        r1 = r2 = m;
        i1 = root;
        i2 = -root;
    }
}

// Reflector I - tau v v^T with v = (1, v1, v2) (v2 = 0 for a 2-element one) that maps the
// column (x0, x1, x2) to (beta, 0, 0), beta = -sign(x0) ||x||. tau = 0 when nothing to do.
template <typename T>
static __device__ void reflector3(T x0, T x1, T x2, T& tau, T& v1, T& v2) {
    const T scale = fabs(x0) + fabs(x1) + fabs(x2);
    tau = v1 = v2 = T(0);
    if (scale == T(0) || (x1 == T(0) && x2 == T(0))) return;
    const T y0 = x0 / scale, y1 = x1 / scale, y2 = x2 / scale;
    const T nrm = sqrt(y0 * y0 + y1 * y1 + y2 * y2);
    const T beta = (y0 > T(0)) ? -nrm : nrm;
    const T den = y0 - beta;
    tau = (beta - y0) / beta;
    v1 = y1 / den;
    v2 = y2 / den;
}

template <typename T>
static __device__ int hess_qr_eigs(T* H, int ld, int d, T* wr, T* wi) {
    const int lane = LANE;
    const T eps = EpsOf<T>::v();
    auto at = [&](int i, int j) -> T& { return H[i + j * ld]; };
    // a norm for windows whose diagonal neighbours are both zero
    T hnorm = T(0);
    for (int i = lane; i < d; i += 32)
        for (int j = (i > 0 ? i - 1 : 0); j < d; ++j) hnorm = fmax(hnorm, fabs(at(i, j)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hnorm = fmax(hnorm, __shfl_xor_sync(0xffffffffu, hnorm, o));
    int hi = d - 1;
    int since_split = 0, budget = 30 * d, failed = 0;
    while (hi >= 0) {
        // bottom-up search for the start of the unreduced window ending at hi
        int lo = hi;
        while (lo > 0) {
            T nb = fabs(at(lo - 1, lo - 1)) + fabs(at(lo, lo));
            if (nb == T(0)) nb = hnorm;
            if (fabs(at(lo, lo - 1)) <= eps * nb) break;
            --lo;
        }
        WSYNC();
        if (lane == 0 && lo > 0) at(lo, lo - 1) = T(0);
        WSYNC();
        const int size = hi - lo + 1;
        if (size <= 2) {
            if (lane == 0) {
                if (size == 1) {
                    wr[hi] = at(hi, hi);
                    wi[hi] = T(0);
                } else {
                    eig2x2(at(lo, lo), at(lo, hi), at(hi, lo), at(hi, hi), wr[lo], wi[lo], wr[hi], wi[hi]);
                }
            }
            hi = lo - 1;
            since_split = 0;
            WSYNC();
            continue;
        }
        if (budget-- <= 0) {
            if (lane == 0)
                for (int i = lo; i <= hi; ++i) { wr[i] = at(i, i); wi[i] = T(0); }
            failed = 1;
            hi = lo - 1;
            WSYNC();
            continue;
        }
        // shift pair through its sum s and product t
        T s, t;
        if (++since_split % 11 == 10) {
            const T mu = at(hi, hi) + T(1.5) * (fabs(at(hi, hi - 1)) + fabs(at(hi - 1, hi - 2)));
            s = T(2) * mu;
            t = mu * mu;
        } else {
            const T p = at(hi - 1, hi - 1), q = at(hi - 1, hi), r = at(hi, hi - 1), w = at(hi, hi);
            s = p + w;
            t = p * w - q * r;
        }
        // first column of H^2 - s H + t I within the window
        T x0 = at(lo, lo) * at(lo, lo) + at(lo, lo + 1) * at(lo + 1, lo) - s * at(lo, lo) + t;
        T x1 = at(lo + 1, lo) * (at(lo, lo) + at(lo + 1, lo + 1) - s);
        T x2 = at(lo + 1, lo) * at(lo + 2, lo + 1);
        for (int c = lo; c <= hi - 1; ++c) {
            const bool two = (c == hi - 1);       // last reflector touches two rows
            T tau, v1, v2;
            reflector3(x0, x1, two ? T(0) : x2, tau, v1, v2);
            WSYNC();
            if (tau != T(0)) {
                const int r2 = two ? c + 1 : c + 2;
                // from the left: rows c..r2, columns max(lo, c-1)..hi
                for (int j = (c > lo ? c - 1 : lo) + lane; j <= hi; j += 32) {
                    T dot = at(c, j) + v1 * at(c + 1, j);
                    if (!two) dot += v2 * at(c + 2, j);
                    dot *= tau;
                    at(c, j) -= dot;
                    at(c + 1, j) -= dot * v1;
                    if (!two) at(c + 2, j) -= dot * v2;
                }
                WSYNC();
                // from the right: columns c..r2, rows lo..min(c+3, hi)
                const int rmax = (c + 3 < hi) ? c + 3 : hi;
                for (int i = lo + lane; i <= rmax; i += 32) {
                    T dot = at(i, c) + v1 * at(i, c + 1);
                    if (!two) dot += v2 * at(i, c + 2);
                    dot *= tau;
                    at(i, c) -= dot;
                    at(i, c + 1) -= dot * v1;
                    if (!two) at(i, c + 2) -= dot * v2;
                }
                (void)r2;
                WSYNC();
            }
            // the entries below the subdiagonal that the reflector just annihilated
            if (lane == 0 && c > lo) {
                at(c + 1, c - 1) = T(0);
                if (!two) at(c + 2, c - 1) = T(0);
            }
            WSYNC();
            if (!two) {
                // the bulge below column c, to be annihilated by the next reflector
                x0 = at(c + 1, c);
                x1 = at(c + 2, c);
                x2 = (c + 3 <= hi) ? at(c + 3, c) : T(0);
            }
        }
        WSYNC();
    }
    WSYNC();
    return failed;
}

// Inverse iteration for the eigenvalue (lr, li) of the Hessenberg matrix Hm (d x d, ld): two
// solves of (Hm - lambda I) x = rhs by Gaussian elimination with partial pivoting between
// adjacent rows. U (workspace, d*(d+1) doubles: packed complex upper triangle) and small
// vectors in smem.
// Result x (complex) in xr, xi, normalised to unit 2-norm.
static __device__ void inv_iter(const double* Hm, int ld, int d, double lr, double li, double hnorm, double* U,
                         double* xr, double* xi, double* mr, double* mi, int* swp, double* cr, double* ci) {
    const int lane = LANE;
    double eps = 1e-14 * (hnorm > 0.0 ? hnorm : 1.0);
    // perturb lambda slightly to avoid an exactly singular system
    lr += eps;
    // rows of U packed upper-triangular: element (i, j >= i) at UP(i, j), complex (re, im)
#define UP(i, j) ((((i) * d - ((i) * ((i) - 1)) / 2) + ((j) - (i))) * 2)
    // cur row (complex) in cr/ci
    for (int j = lane; j < d; j += 32) {
        cr[j] = Hm[0 + j * ld] - (j == 0 ? lr : 0.0);
        ci[j] = (j == 0 ? -li : 0.0);
    }
    WSYNC();
    for (int k = 0; k < d - 1; ++k) {
        // next row k+1 of (H - lambda I), nonzero from column k
        double nr_k = Hm[(k + 1) + k * ld];
        double ni_k = 0.0;
        double ar = cr[k], ai = ci[k];
        bool sw = (fabs(nr_k) + fabs(ni_k)) > (fabs(ar) + fabs(ai));
        // pivot row p = sw ? next : cur; other row o
        // l = o[k] / p[k]
        double pr = sw ? nr_k : ar, pi = sw ? ni_k : ai;
        double orr = sw ? ar : nr_k, oi = sw ? ai : ni_k;
        double den = pr * pr + pi * pi;
        if (den == 0.0) { pr = eps; pi = 0.0; den = eps * eps; }
        const double iden = 1.0 / den;
        double lre = (orr * pr + oi * pi) * iden, lim = (oi * pr - orr * pi) * iden;
        if (lane == 0) { mr[k] = lre; mi[k] = lim; swp[k] = sw ? 1 : 0; }
        for (int j = k + lane; j < d; j += 32) {
            double hr = Hm[(k + 1) + j * ld] - ((j == k + 1) ? lr : 0.0);
            double hi = (j == k + 1) ? -li : 0.0;
            double pjr = sw ? hr : cr[j], pji = sw ? hi : ci[j];
            double ojr = sw ? cr[j] : hr, oji = sw ? ci[j] : hi;
            if (j == k) { pjr = pr; pji = pi; }
            U[UP(k, j)] = pjr;
            U[UP(k, j) + 1] = pji;
            // new current row = other - l * pivot
            double nr2 = ojr - (lre * pjr - lim * pji);
            double ni2 = oji - (lre * pji + lim * pjr);
            cr[j] = nr2;
            ci[j] = ni2;
        }
        WSYNC();
    }
    if (lane == 0) {
        double ur = cr[d - 1], ui = ci[d - 1];
        if (ur == 0.0 && ui == 0.0) ur = eps;
        U[UP(d - 1, d - 1)] = ur;
        U[UP(d - 1, d - 1) + 1] = ui;
    }
    WSYNC();
    for (int i = lane; i < d; i += 32) { xr[i] = 1.0; xi[i] = 0.0; }
    WSYNC();
    for (int pass = 0; pass < 2; ++pass) {
        // forward: apply the recorded swaps/multipliers to the rhs
        if (lane == 0) {
            for (int k = 0; k < d - 1; ++k) {
                double ar = xr[k], ai = xi[k], br = xr[k + 1], bi = xi[k + 1];
                if (swp[k]) { double tr = ar, ti = ai; ar = br; ai = bi; br = tr; bi = ti; }
                xr[k] = ar; xi[k] = ai;
                xr[k + 1] = br - (mr[k] * ar - mi[k] * ai);
                xi[k + 1] = bi - (mr[k] * ai + mi[k] * ar);
            }
        }
        WSYNC();
        // back substitution with U
        for (int i = d - 1; i >= 0; --i) {
            double sr = 0.0, si = 0.0;
            for (int j = i + 1 + lane; j < d; j += 32) {
                double ur = U[UP(i, j)], ui = U[UP(i, j) + 1];
                sr += ur * xr[j] - ui * xi[j];
                si += ur * xi[j] + ui * xr[j];
            }
            sr = wsum(sr);
            si = wsum(si);
            if (lane == 0) {
                double br = xr[i] - sr, bi = xi[i] - si;
                double ur = U[UP(i, i)], ui = U[UP(i, i) + 1];
                const double iden = 1.0 / (ur * ur + ui * ui);
                xr[i] = (br * ur + bi * ui) * iden;
                xi[i] = (bi * ur - br * ui) * iden;
            }
            WSYNC();
        }
        double nrm = 0.0;
        for (int i = lane; i < d; i += 32) nrm += xr[i] * xr[i] + xi[i] * xi[i];
        nrm = sqrt(wsum(nrm));
        double inv = (nrm > 0.0 && nrm < 1e300) ? 1.0 / nrm : 0.0;
        for (int i = lane; i < d; i += 32) { xr[i] *= inv; xi[i] *= inv; }
        WSYNC();
    }
#undef UP
}

// Selection of the k eigenvalues of smallest |theta| (largest == 0) or largest |mu|
// (largest == 1), with the conjugate-pair rule: a pair split at the boundary is taken whole
// if k + 1 < mcap and k + 1 <= d, dropped otherwise. sel[] receives indices (a pair is
// represented by its member with wi > 0). Returns the number of basis columns.
static __device__ int select_eigs(const double* wr, const double* wi, int d, int k, int largest, int mcap, int* sel,
                           int* nsel) {
    // insertion-sort indices by the key (stable)
    int order[SM_DMAX];
    for (int i = 0; i < d; ++i) order[i] = i;
    auto key = [&](int i) {
        double mgn = hypot(wr[i], wi[i]);
        if (!(mgn == mgn)) return largest ? -1.0 : 1e308;
        return largest ? -mgn : mgn;
    };
    for (int i = 1; i < d; ++i) {
        int v = order[i];
        double kv = key(v);
        int j = i - 1;
        while (j >= 0 && key(order[j]) > kv) { order[j + 1] = order[j]; --j; }
        order[j + 1] = v;
    }
    int kk = min(k, d);
    // chosen = first kk in order; pair rule for the last
    bool chosen[SM_DMAX];
    for (int i = 0; i < d; ++i) chosen[i] = false;
    for (int i = 0; i < kk; ++i) chosen[order[i]] = true;
    if (kk > 0) {
        int last = order[kk - 1];
        if (wi[last] != 0.0) {
            int partner = -1;
            for (int i = 0; i < d; ++i)
                if (i != last && wr[i] == wr[last] && wi[i] == -wi[last]) { partner = i; break; }
            if (partner >= 0 && !chosen[partner]) {
                if (kk + 1 < mcap && kk + 1 <= d && kk + 1 <= SM_KMAX) chosen[partner] = true;
                else chosen[last] = false;
            }
        }
    }
    int cnt = 0, cols = 0;
    for (int t = 0; t < d; ++t) {
        int i = order[t];
        if (!chosen[i]) continue;
        if (wi[i] == 0.0) { sel[cnt++] = i; cols += 1; }
        else if (wi[i] > 0.0) { sel[cnt++] = i; cols += 2; }
        else {
            // member with wi < 0: represented by its partner (wi > 0) if that one is chosen
            bool has = false;
            for (int q = 0; q < d; ++q)
                if (q != i && wr[q] == wr[i] && wi[q] == -wi[i] && chosen[q]) has = true;
            if (!has) { sel[cnt++] = i; cols += 2; }
        }
    }
    *nsel = cnt;
    return cols;
}

// Eigenvalues and selection (one warp): Householder reduction of M (d x d, ld d, FP64, in place)
// to Hessenberg form with the similarity accumulated in Qh (global, ld d); eigenvalues by the
// double-shift Hessenberg QR iteration on a copy in `work` (d*d doubles of shared memory): in FP32
// on a power-of-two scaled copy (eig64 == 0), or in FP64 (eig64 != 0); the selected eigenvalues
// in sel[0..nsel) with the first basis column of each in colofs[]. Returns the number of columns.
static __device__ int eig_values(double* M, double* work, int eig64, int d, int k, int largest, int mcap, double* Qh,
                          double* wr, double* wi, double* vec, int* sel, int* colofs, int* nsel_out, double* hn_out,
                          int* fail_out) {
    const int lane = LANE;
    __shared__ float wrf[SM_DMAX], wif[SM_DMAX];
    __shared__ int nsel_s, cols_s;
    hess_reduce(M, d, d, Qh, vec);
    double hn = 0.0;
    for (int e = lane; e < d * d; e += 32) hn = fmax(hn, fabs(M[e]));
    hn = warp_max(hn);
    if (eig64) {
        for (int e = lane; e < d * d; e += 32) work[e] = M[e];
        WSYNC();
        *fail_out = hess_qr_eigs<double>(work, d, d, wr, wi);
    } else {
        // scale by 2^-e with hn 2^-e in [0.5, 1): no FP32 overflow, and the unscaling is exact
        float* Af = reinterpret_cast<float*>(work);
        int ex = 0;
        if (hn > 0.0 && hn < 1.7976931348623157e308) frexp(hn, &ex);
        const double sc = ldexp(1.0, -ex);
        for (int e = lane; e < d * d; e += 32) Af[e] = (float)(M[e] * sc);
        WSYNC();
        *fail_out = hess_qr_eigs<float>(Af, d, d, wrf, wif);
        for (int i = lane; i < d; i += 32) {
            wr[i] = (double)wrf[i] / sc;
            wi[i] = (double)wif[i] / sc;
        }
    }
    WSYNC();
    if (lane == 0) {
        int ns;
        cols_s = select_eigs(wr, wi, d, k, largest, mcap, sel, &ns);
        nsel_s = ns;
        int c = 0;
        for (int t = 0; t < ns; ++t) {
            colofs[t] = c;
            c += (wi[sel[t]] != 0.0) ? 2 : 1;
        }
    }
    WSYNC();
    *nsel_out = nsel_s;
    *hn_out = hn;
    return cols_s;
}

// Doubles of shared workspace per warp for eig_vectors.
__host__ __device__ inline int eigvec_stride(int d) { return d * (d + 1) + 7 * d; }

// Eigenvectors of the selected eigenvalues (all warps of the CTA, nw of them with a workspace
// each in wbuf): FP64 inverse iteration on the Hessenberg matrix M from the eigenvalue as shift,
// then z = Qh x into the real basis P (d x cols, ld ldp): a real eigenvalue gives one column, a
// conjugate pair the real and imaginary parts.
static __device__ void eig_vectors(const double* M, int d, const double* Qh, double* P, int ldp, const double* wr,
                            const double* wi, const int* sel, const int* colofs, int nsel, double hn, double* wbuf,
                            int nw) {
    const int lane = LANE, warp = threadIdx.x >> 5;
    if (warp >= nw) return;
    double* U = wbuf + (size_t)warp * eigvec_stride(d);
    double* xr = U + d * (d + 1);
    double* xi = xr + d;
    double* mr = xi + d;
    double* mi = mr + d;
    double* cr = mi + d;
    double* ci = cr + d;
    int* swp = reinterpret_cast<int*>(ci + d);
    for (int t = warp; t < nsel; t += nw) {
        const int i = sel[t];
        const double lr = wr[i], li = fabs(wi[i]);
        inv_iter(M, d, d, lr, li, hn, U, xr, xi, mr, mi, swp, cr, ci);
        const int col = colofs[t];
        for (int r = lane; r < d; r += 32) {
            double zr = 0.0, zi = 0.0;
            for (int c = 0; c < d; ++c) {
                const double q = Qh[r + c * d];
                zr += q * xr[c];
                zi += q * xi[c];
            }
            P[r + col * ldp] = zr;
            if (li != 0.0) P[r + (col + 1) * ldp] = zi;
        }
        WSYNC();
    }
}

// ------------------------------------------------------------------ cycle end
// Dynamic shared memory layout: M [(d+1)*d], Wk [2*d*d + 4*d] (G / hqr copy / inverse-iteration rows).
constexpr int CLOSE_THREADS = 128;
constexpr int CLOSE_SMEM_DOUBLES = 210 * 1024 / 8;

// Warps that get an inverse-iteration workspace behind the (d+1) x d block M in a shared
// workspace of avail_doubles doubles.
__host__ __device__ inline int eigvec_warps(int d, int mrows, int avail_doubles) {
    const int avail = avail_doubles - mrows * d;
    int nw = avail / eigvec_stride(d);
    nw = nw > CLOSE_THREADS / 32 ? CLOSE_THREADS / 32 : nw;
    return nw < 1 ? 1 : nw;
}

// The four warps 0..3 of the calling CTA synchronise on named barrier 1, so a larger CTA (the
// persistent batch kernel) can run the cycle end on its first 128 threads.
__device__ __forceinline__ void close_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Warp 0 runs everything but the eigenvectors, which all warps share (one selected eigenvalue
// each at a time: GB300's FP64 pipes are per SM sub-partition, so four warps are four times one).
// smem: smem_doubles doubles of shared workspace. Called by exactly the CLOSE_THREADS threads of
// warps 0..3.
static __device__ void cycle_close_dev(SmallState* st, double* Qh, double* Pbuf, double* Gq, double* smem,
                                int smem_doubles) {
    const int lane = LANE, warp = threadIdx.x >> 5;
    const int j = st->j, kc = st->kc, d = kc + j;
    const int first = st->first;
    double* M = smem;                          // (d+1) x d, ld d+1
    double* Wk = smem + (size_t)(d + 1) * d;   // (d+1) x d doubles; the eigenvector workspaces from here
    __shared__ double y[SM_DMAX], tau[SM_DMAX + 1], wr[SM_DMAX], wi[SM_DMAX], vec[SM_DMAX + 1];
    __shared__ int sel[SM_DMAX], colofs[SM_DMAX];
    __shared__ int nsel_s, cols_s;
    __shared__ double hn_s;
    const int k = st->k_target;
    const bool recycle = (k > 0) && (first ? (j > k) : true) && d >= 1;

    if (warp == 0) {
    // D_k = diag(1 / ||u_i||) from the Gram matrix U^T U (ld kc)
    for (int i = lane; i < kc; i += 32) st->dk[i] = 1.0 / sqrt(st->UtU[i + i * kc]);
    WSYNC();
    // ---- least squares: y2 = Hr(0:j,0:j)^-1 g(0:j) (Givens form), y1 = -D^-1 B y2
    if (lane == 0) {
        for (int i = j - 1; i >= 0; --i) {
            double s = st->g[i];
            for (int c = i + 1; c < j; ++c) s -= st->Hr[i + c * SM_LDH] * y[kc + c];
            y[kc + i] = s / st->Hr[i + i * SM_LDH];
        }
        for (int i = 0; i < kc; ++i) {
            double s = 0.0;
            for (int c = 0; c < j; ++c) s += st->B[i + c * SM_KMAX] * y[kc + c];
            y[i] = -s / st->dk[i];
        }
    }
    WSYNC();
    // ycoef: [D y1 ; y2] for d += [U V_j] ycoef
    for (int i = lane; i < d; i += 32) st->ycoef[i] = (i < kc) ? st->dk[i] * y[i] : y[i];
    // zcoef: first cycle: beta e1 - H y ; otherwise G y = [D y1 + B y2 ; H y2]
    for (int i = lane; i < d + 1; i += 32) {
        double s;
        if (i < kc) {
            s = st->dk[i] * y[i];
            for (int c = 0; c < j; ++c) s += st->B[i + c * SM_KMAX] * y[kc + c];
        } else {
            int ih = i - kc;
            s = 0.0;
            for (int c = max(ih - 1, 0); c < j; ++c) s += st->H[ih + c * SM_LDH] * y[kc + c];
        }
        st->zcoef[i] = first ? (((i == 0) ? st->beta : 0.0) - s) : s;
    }
    WSYNC();

    if (recycle) {
        // ---- harmonic Ritz matrix M (d x d, ld d)
        if (first) {
            // M = H_j + h^2 f e_j^T with H_j^T f = e_j (Gaussian elimination with partial pivoting)
            // A = H_j^T in Wk (d x d, ld d); rhs e_j in vec
            for (int e = lane; e < d * d; e += 32) {
                int r = e % d, c = e / d;
                Wk[e] = st->H[c + r * SM_LDH];
            }
            for (int i = lane; i < d; i += 32) vec[i] = (i == d - 1) ? 1.0 : 0.0;
            WSYNC();
            for (int c = 0; c < d; ++c) {
                // pivot
                int p = c;
                double best = fabs(Wk[c + c * d]);
                for (int r = c + 1; r < d; ++r)
                    if (fabs(Wk[r + c * d]) > best) { best = fabs(Wk[r + c * d]); p = r; }
                if (p != c) {
                    for (int cc = lane; cc < d; cc += 32) {
                        double tmp = Wk[c + cc * d]; Wk[c + cc * d] = Wk[p + cc * d]; Wk[p + cc * d] = tmp;
                    }
                    WSYNC();
                    if (lane == 0) { double tmp = vec[c]; vec[c] = vec[p]; vec[p] = tmp; }
                }
                WSYNC();
                double piv = Wk[c + c * d];
                if (piv == 0.0) piv = 1e-300;
                for (int r = c + 1 + lane; r < d; r += 32) {
                    double l = Wk[r + c * d] / piv;
                    for (int cc = c + 1; cc < d; ++cc) Wk[r + cc * d] -= l * Wk[c + cc * d];
                    vec[r] -= l * vec[c];
                }
                WSYNC();
            }
            if (lane == 0) {
                for (int r = d - 1; r >= 0; --r) {
                    double s = vec[r];
                    for (int cc = r + 1; cc < d; ++cc) s -= Wk[r + cc * d] * vec[cc];
                    double piv = Wk[r + r * d];
                    vec[r] = s / (piv != 0.0 ? piv : 1e-300);
                }
            }
            WSYNC();
            const double h = st->H[j + (j - 1) * SM_LDH];
            for (int e = lane; e < d * d; e += 32) {
                int r = e % d, c = e / d;
                double v = st->H[r + c * SM_LDH];
                if (c == d - 1) v += h * h * vec[r];
                M[e] = v;
            }
            WSYNC();
        } else {
            // G ((d+1) x d, ld d+1) in Wk; W^T V ((d+1) x d, ld d+1) in M
            const int ldg = d + 1;
            for (int e = lane; e < ldg * d; e += 32) {
                int r = e % ldg, c = e / ldg;
                double gv, wv;
                if (r < kc) {
                    gv = (c < kc) ? ((r == c) ? st->dk[r] : 0.0) : st->B[r + (c - kc) * SM_KMAX];
                    wv = (c < kc) ? st->WtU[r + c * SM_LDG] * st->dk[c] : 0.0;
                } else {
                    int ih = r - kc;
                    gv = (c < kc) ? 0.0 : st->H[ih + (c - kc) * SM_LDH];
                    wv = (c < kc) ? st->WtU[r + c * SM_LDG] * st->dk[c] : ((ih == c - kc) ? 1.0 : 0.0);
                }
                Wk[e] = gv;
                M[e] = wv;
            }
            WSYNC();
            house_qr(Wk, ldg, ldg, d, tau);
            house_apply_qt(Wk, ldg, ldg, d, tau, M, ldg, d);
            // M(0:d, :) = R_G^-1 M(0:d, :)
            for (int c = lane; c < d; c += 32) {
                for (int r = d - 1; r >= 0; --r) {
                    double s = M[r + c * ldg];
                    for (int q = r + 1; q < d; ++q) s -= Wk[r + q * ldg] * M[q + c * ldg];
                    double piv = Wk[r + r * ldg];
                    M[r + c * ldg] = s / (piv != 0.0 ? piv : 1e-300);
                }
            }
            WSYNC();
            // compact to ld d
            for (int c = 0; c < d; ++c) {
                for (int r = lane; r < d; r += 32) vec[r] = M[r + c * ldg];
                WSYNC();
                for (int r = lane; r < d; r += 32) M[r + c * d] = vec[r];
                WSYNC();
            }
        }
        int fail = 0, nsel = 0;
        double hn = 0.0;
        const int cols = eig_values(M, Wk, st->eig64, d, k, first ? 0 : 1, st->m, Qh, wr, wi, vec, sel, colofs,
                                    &nsel, &hn, &fail);
        // non-converged eigenvalues keep their diagonal estimates (fail is not an error)
        if (lane == 0) {
            nsel_s = nsel;
            cols_s = cols;
            hn_s = hn;
        }
        for (int i = lane; i < d; i += 32) { st->eig_wr[i] = wr[i]; st->eig_wi[i] = wi[i]; }
    }
    }  // warp 0
    close_bar();
    if (recycle)
        eig_vectors(M, d, Qh, Pbuf, d, wr, wi, sel, colofs, nsel_s, hn_s, Wk, eigvec_warps(d, d + 1, smem_doubles));
    close_bar();
    if (warp != 0) return;
    int knew = 0;
    if (recycle) {
        int cols = cols_s;
        // ---- G P ((d+1) x cols) in Gq (global), QR with positive diagonal, rank drop
        const int ldg = d + 1;
        for (int e = lane; e < ldg * cols; e += 32) {
            int r = e % ldg, c = e / ldg;
            double s = 0.0;
            for (int q = 0; q < d; ++q) {
                double gv;
                if (r < kc) gv = (q < kc) ? ((r == q) ? st->dk[r] : 0.0) : st->B[r + (q - kc) * SM_KMAX];
                else {
                    int ih = r - kc;
                    gv = (q < kc) ? 0.0 : st->H[ih + (q - kc) * SM_LDH];
                }
                s += gv * Pbuf[q + c * d];
            }
            Gq[e] = s;
        }
        WSYNC();
        // Householder QR of Gq in Wk copy (ld ldg)
        for (int e = lane; e < ldg * cols; e += 32) Wk[e] = Gq[e];
        WSYNC();
        house_qr(Wk, ldg, ldg, cols, tau);
        // rank: keep columns with |R_ii| > 1e-12 max |R_jj| (columns are kept in order; a
        // dropped column is removed from P and the QR recomputed)
        __shared__ int keep_s[SM_KMAX + 2];
        __shared__ int nk_s;
        if (lane == 0) {
            double mx = 0.0;
            for (int i = 0; i < cols; ++i) mx = fmax(mx, fabs(Wk[i + i * ldg]));
            int nk = 0;
            for (int i = 0; i < cols; ++i) {
                bool ok = fabs(Wk[i + i * ldg]) > 1e-12 * mx;
                keep_s[i] = ok;
                nk += ok;
            }
            nk_s = nk;
        }
        WSYNC();
        int nk = nk_s;
        if (nk < cols) {
            // compact P and Gq columns, redo QR
            if (lane == 0) {
                int w2 = 0;
                for (int c = 0; c < cols; ++c) {
                    if (!keep_s[c]) continue;
                    for (int r = 0; r < d; ++r) Pbuf[r + w2 * d] = Pbuf[r + c * d];
                    for (int r = 0; r < ldg; ++r) Gq[r + w2 * ldg] = Gq[r + c * ldg];
                    ++w2;
                }
            }
            WSYNC();
            cols = nk;
            for (int e = lane; e < ldg * cols; e += 32) Wk[e] = Gq[e];
            WSYNC();
            house_qr(Wk, ldg, ldg, cols, tau);
        }
        // Q explicit into M ((d+1) x cols, ld ldg) ; R in Wk upper triangle
        house_form_q(Wk, ldg, ldg, cols, tau, M, ldg, cols);
        // signs: make R_ii >= 0
        for (int c = lane; c < cols; c += 32) {
            if (Wk[c + c * ldg] < 0.0) {
                for (int r = 0; r < ldg; ++r) M[r + c * ldg] = -M[r + c * ldg];
                for (int q = c; q < cols; ++q) Wk[c + q * ldg] = -Wk[c + q * ldg];
            }
        }
        WSYNC();
        // Ccoef = Q
        for (int e = lane; e < ldg * cols; e += 32) {
            int r = e % ldg, c = e / ldg;
            st->Ccoef[r + c * SM_LDG] = M[e];
        }
        // Ucoef = diag(D, I) P R^-1 : solve X R = P  (row-wise forward substitution over columns)
        for (int r = lane; r < d; r += 32) {
            double dscale = (r < kc) ? st->dk[r] : 1.0;
            for (int c = 0; c < cols; ++c) {
                double s = Pbuf[r + c * d];
                for (int q = 0; q < c; ++q) s -= st->Ucoef[r + q * SM_LDG] / dscale * Wk[q + c * ldg];
                st->Ucoef[r + c * SM_LDG] = dscale * s / Wk[c + c * ldg];
            }
        }
        WSYNC();
        knew = cols;
    }
    if (lane == 0) st->knew = knew;
}

// ------------------------------------------------------------------ Cholesky of a Gram matrix
// G2 (k x k, ld k) = R^T R; Rinv = R^-1 accumulated: Rinv <- Rinv_prev * R^-1 when
// accumulate != 0 (Cholesky QR twice). knew = k, or 0 if the Gram matrix is not positive definite.
// One thread (also called from the persistent batch kernel).
static __device__ void chol_gram_dev(SmallState* st, int k, int accumulate) {
    if (accumulate && st->knew == 0) return;  // the first Cholesky already failed
    double* G = st->G2;
    const int ldg = k;
    // in-place Cholesky (upper R stored in G's upper triangle), column-major ld k
    for (int c = 0; c < k; ++c) {
        for (int r = 0; r <= c; ++r) {
            double s = G[r + c * ldg];
            for (int q = 0; q < r; ++q) s -= G[q + r * ldg] * G[q + c * ldg];
            if (r == c) {
                if (!(s > 0.0)) { st->knew = 0; return; }
                G[r + c * ldg] = sqrt(s);
            } else {
                G[r + c * ldg] = s / G[r + r * ldg];
            }
        }
    }
    // Rnew^-1 (upper) by back substitution, column by column
    double* T = st->Ucoef;  // scratch k x k (ld SM_LDG)
    for (int c = 0; c < k; ++c) {
        for (int r = c; r >= 0; --r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int q = r + 1; q <= c; ++q) s -= G[r + q * ldg] * T[q + c * SM_LDG];
            T[r + c * SM_LDG] = s / G[r + r * ldg];
        }
        for (int r = c + 1; r < k; ++r) T[r + c * SM_LDG] = 0.0;
    }
    if (!accumulate) {
        for (int c = 0; c < k; ++c)
            for (int r = 0; r < k; ++r) st->Rinv[r + c * SM_KMAX] = T[r + c * SM_LDG];
    } else {
        // Rinv = Rinv * T
        double tmp[SM_KMAX];
        for (int r = 0; r < k; ++r) {
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int q = 0; q < k; ++q) s += st->Rinv[r + q * SM_KMAX] * T[q + c * SM_LDG];
                tmp[c] = s;
            }
            for (int c = 0; c < k; ++c) st->Rinv[r + c * SM_KMAX] = tmp[c];
        }
    }
    // Ccoef = T (the factor applied to Z to get the orthonormal columns this round)
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) st->Ccoef[r + c * SM_LDG] = T[r + c * SM_LDG];
    st->knew = k;
}

// ------------------------------------------------------------------ standalone eigen test
// ------------------------------------------------------------------ kernels and launchers
// Left out when another translation unit includes this file for the device functions alone
// (the persistent batch kernel, which is not built with separate device linking).
#ifndef GIR_SMALL_DEVICE_ONLY

__global__ void k_givens_step(SmallState* st) {
    if (threadIdx.x == 0) givens_step_dev(st);
}

gir_status launch_givens_step(SmallState* st, cudaStream_t s) {
    count_launch(), k_givens_step<<<1, 32, 0, s>>>(st);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

// ------------------------------------------------------------------ scale kernel
__global__ void k_scale_by(double* __restrict__ w, int64_t n, const double* __restrict__ factor, int invert,
                           int round32) {
    double f = *factor;
    if (invert) f = (f != 0.0) ? 1.0 / f : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = w[i] * f;
        if (round32) v = (double)__double2float_rn(v);
        w[i] = v;
    }
}

gir_status launch_scale_by(double* w, int64_t n, const double* factor, int invert, int round32, cudaStream_t s) {
    int g = (int)gmin<int64_t>((n + 255) / 256, 1024);
    count_launch(), k_scale_by<<<g, 256, 0, s>>>(w, n, factor, invert, round32);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

__global__ void __launch_bounds__(CLOSE_THREADS) k_cycle_close(SmallState* st, double* Qh, double* Pbuf, double* Gq) {
    extern __shared__ double smem[];
    cycle_close_dev(st, Qh, Pbuf, Gq, smem, CLOSE_SMEM_DOUBLES);
}

gir_status launch_cycle_close(SmallState* st, double* qh_scratch, cudaStream_t s) {
    static std::atomic<unsigned> attr_done{0};
    const size_t smem = (size_t)CLOSE_SMEM_DOUBLES * 8;
    GIR_CUDA_TRY(ensure_dyn_smem((const void*)k_cycle_close, (int)smem, attr_done));
    double* Qh = qh_scratch;
    double* Pbuf = qh_scratch + SM_DMAX * SM_DMAX;
    double* Gq = Pbuf + SM_DMAX * (SM_KMAX + 2);
    count_launch(), k_cycle_close<<<1, CLOSE_THREADS, smem, s>>>(st, Qh, Pbuf, Gq);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

__global__ void k_chol_gram(SmallState* st, int k, int accumulate) {
    if (threadIdx.x == 0) chol_gram_dev(st, k, accumulate);
}

gir_status launch_chol_gram(SmallState* st, int k, cudaStream_t s) {
    // accumulate flag encoded in the sign of k
    int acc = k < 0;
    count_launch(), k_chol_gram<<<1, 32, 0, s>>>(st, acc ? -k : k, acc);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

__global__ void __launch_bounds__(CLOSE_THREADS) k_small_eig(const double* Min, int d, int k, int largest, int mcap,
                                                             int eig64, double* wr_o, double* wi_o, double* P,
                                                             int* kout, double* Qh) {
    extern __shared__ double smem[];
    const int lane = LANE, warp = threadIdx.x >> 5;
    double* M = smem;
    double* Wk = smem + (size_t)(d + 1) * d;
    __shared__ double wr[SM_DMAX], wi[SM_DMAX], vec[SM_DMAX + 1];
    __shared__ int sel[SM_DMAX], colofs[SM_DMAX];
    __shared__ int nsel_s, cols_s, fail_s;
    __shared__ double hn_s;
    if (warp == 0) {
        for (int e = lane; e < d * d; e += 32) M[e] = Min[e];
        WSYNC();
        int fail = 0, nsel = 0;
        double hn = 0.0;
        const int cols = eig_values(M, Wk, eig64, d, k, largest, mcap, Qh, wr, wi, vec, sel, colofs, &nsel, &hn,
                                    &fail);
        if (lane == 0) {
            nsel_s = nsel;
            cols_s = cols;
            hn_s = hn;
            fail_s = fail;
        }
    }
    __syncthreads();
    eig_vectors(M, d, Qh, P, d, wr, wi, sel, colofs, nsel_s, hn_s, Wk, eigvec_warps(d, d + 1, CLOSE_SMEM_DOUBLES));
    __syncthreads();
    if (warp != 0) return;
    for (int i = lane; i < d; i += 32) { wr_o[i] = wr[i]; wi_o[i] = wi[i]; }
    if (lane == 0) *kout = fail_s ? -cols_s - 1 : cols_s;
}

gir_status launch_small_eig(const double* M, int d, int k, int largest, int mcap, int eig64, double* wr, double* wi,
                            double* P, int kcap, int* kout, double* scratch, cudaStream_t s) {
    (void)kcap;
    static std::atomic<unsigned> attr_done{0};
    const size_t smem = (size_t)CLOSE_SMEM_DOUBLES * 8;
    GIR_CUDA_TRY(ensure_dyn_smem((const void*)k_small_eig, (int)smem, attr_done));
    count_launch(), k_small_eig<<<1, CLOSE_THREADS, smem, s>>>(M, d, k, largest, mcap, eig64, wr, wi, P, kout,
                                                                  scratch);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

#endif  // GIR_SMALL_DEVICE_ONLY

}  // namespace gir
