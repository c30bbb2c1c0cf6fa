// Host-side validation of a problem and construction of the FP32 tables the
// kernels read (shared by the single-problem, batched and allocation-free
// entry points).
#pragma once
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/empc.h"
#include "empc_internal.h"

namespace empc {

inline bool all_finite(const double* v, size_t k) {
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Checks the arguments of one problem; returns EMPC_OK or a status with msg.
// Q and R may be dense: only their symmetric parts enter the cost (x'Qx =
// x' (Q + Q')/2 x), which must be positive semidefinite (checked when the
// tables are built).
inline empc_status validate_problem(const double* A, const double* B, const double* Q,
                                    const double* R, const double* bounds, int n, int m,
                                    int horizon, int knots, int pop, std::string& msg) {
    if (!A || !B || !Q || !R || !bounds) return msg = "NULL model pointer", EMPC_EINVAL;
    if (n < 1 || n > 128 || m < 1 || m > 128)
        return msg = "need 1 <= n <= 128 and 1 <= m <= 128", EMPC_EINVAL;
    if (horizon < 1 || knots < 1 || knots > horizon)
        return msg = "need horizon >= 1 and 1 <= knots <= horizon", EMPC_EINVAL;
    if (pop < 1 || pop > 32768) return msg = "need 1 <= pop <= 32768", EMPC_EINVAL;
    if (!all_finite(A, (size_t)n * n) || !all_finite(B, (size_t)n * m) ||
        !all_finite(Q, (size_t)n * n) || !all_finite(R, (size_t)m * m) ||
        !all_finite(bounds, (size_t)m * 2))
        return msg = "non-finite model, weight or bound", EMPC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (Q[(size_t)i * n + i] < 0.0) return msg = "Q must be >= 0", EMPC_EINVAL;
    for (int i = 0; i < m; ++i) {
        if (R[(size_t)i * m + i] < 0.0) return msg = "R must be >= 0", EMPC_EINVAL;
        if (!(bounds[2 * i] <= bounds[2 * i + 1])) return msg = "need u_min <= u_max", EMPC_EINVAL;
    }
    return EMPC_OK;
}

// Whether the symmetric part of the k x k matrix M has a non-zero entry off
// its diagonal.
inline bool has_off_diagonal(const double* M, int k) {
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j)
            if (i != j && 0.5 * (M[(size_t)i * k + j] + M[(size_t)j * k + i]) != 0.0) return true;
    return false;
}

// Symmetric eigendecomposition S = V diag(S_ii after the call) V' by cyclic
// Jacobi rotations (Golub & Van Loan, Matrix Computations, Sec. 8.5): each
// rotation zeroes one off-diagonal pair; sweeps repeat until the off-diagonal
// mass is at rounding level.  S (k x k, row-major) is overwritten; V (k x k,
// row-major, columns = eigenvectors) is written.  No allocation.
inline void jacobi_eigen(double* S, double* V, int k) {
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) V[(size_t)i * k + j] = i == j ? 1.0 : 0.0;
    double fro = 0.0;
    for (size_t t = 0; t < (size_t)k * k; ++t) fro += S[t] * S[t];
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) off += S[(size_t)i * k + j] * S[(size_t)i * k + j];
        if (off <= 1e-32 * fro) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double spq = S[(size_t)p * k + q];
                if (spq == 0.0) continue;
                const double theta = (S[(size_t)q * k + q] - S[(size_t)p * k + p]) / (2.0 * spq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) /
                                 (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {
                    if (r == p || r == q) continue;
                    const double srp = S[(size_t)r * k + p], srq = S[(size_t)r * k + q];
                    S[(size_t)r * k + p] = S[(size_t)p * k + r] = c * srp - s * srq;
                    S[(size_t)r * k + q] = S[(size_t)q * k + r] = s * srp + c * srq;
                }
                S[(size_t)p * k + p] -= t * spq;
                S[(size_t)q * k + q] += t * spq;
                S[(size_t)p * k + q] = S[(size_t)q * k + p] = 0.0;
                for (int r = 0; r < k; ++r) {
                    const double vrp = V[(size_t)r * k + p], vrq = V[(size_t)r * k + q];
                    V[(size_t)r * k + p] = c * vrp - s * vrq;
                    V[(size_t)r * k + q] = s * vrp + c * vrq;
                }
            }
    }
}

// Where fill_tables writes one problem's tables.  Every array is provided by
// the caller (sizes in brackets); nothing is allocated, so the
// allocation-free entry point can point these into fixed arrays.
struct TableOut {
    float* D;       // [n][n]  D = A_d - I in the rollout coordinates
    float* BT;      // [m][n]  B_d transposed, rollout coordinates
    float* qd;      // [n]     diagonal state weights (eigenvalues of Q when rotated)
    float* rd;      // [m]     diag(R) (unused when R is dense)
    float* lo;      // [m]     u_min (may be null)
    float* hi;      // [m]     u_max (may be null)
    float* gram;    // [2p]    W_aa, W_a,a+1
    KnotStep* ks;   // [T]
    float* rmat;    // [m][m]  symmetric part of R, written when R is not diagonal
    double* Vt;     // [n][n]  x -> z rotation (row i = eigenvector i of Q), written when rotated
    double* w0;     // [T]     knot weights in FP64
    double* w1;     // [T]
    int* idx;       // [T]     first knot of each step
    double* work;   // [3 n^2 + m^2 + 2p] scratch
};

inline size_t table_work_doubles(int n, int m, int p) {
    return 3 * (size_t)n * n + (size_t)m * m + 2 * (size_t)p;
}

// FP32 tables of one problem.
//  * Knot table of Sec. IV-C in exact integers: idx1 = min(floor(k (p-1) /
//    (T-1)), p-2), c = (k (p-1) - idx1 (T-1)) / (T-1), weights exact
//    rationals rounded once to FP32 (p == 1 or T == 1: constant input).
//  * Gram of the weights: sum_k u_k' R u_k = sum_ij R_ij U_i' W U_j with W
//    tridiagonal, W_aa = sum_k w_ka^2, W_a,a+1 = sum_k w_ka w_k,a+1.
//  * The state cost (x-g)' Q (x-g) of Eq. mpc_problem.  With Q diagonal the
//    rollouts run in the model's own coordinates.  Otherwise its symmetric
//    part is diagonalized, Q_s = V diag(lambda) V', and the rollouts run in
//    z = V' x: z_{k+1} = V'A V z_k + V'B u_k with cost (z - V'g)' diag(lambda)
//    (z - V'g), the same J for every knot vector; the caller rotates x0, the
//    goal and any disturbance with Vt = V'.
// Returns EMPC_EINVAL (with *msg) when Q_s or R_s is not positive
// semidefinite.
inline empc_status fill_tables(const double* A, const double* B, const double* Q,
                               const double* R, const double* bounds, int n, int m, int T,
                               int p, const TableOut& o, bool* rotated, bool* dense_r,
                               const char** msg) {
    const bool rot = has_off_diagonal(Q, n);
    const bool dr = has_off_diagonal(R, m);
    *rotated = rot;
    *dense_r = dr;
    double* S = o.work;                       // [n][n]
    double* V = S + (size_t)n * n;            // [n][n]
    double* Tm = V + (size_t)n * n;           // [n][n]
    double* Rs = Tm + (size_t)n * n;          // [m][m]
    double* Wd = Rs + (size_t)m * m;          // [p]
    double* Wo = Wd + p;                      // [p]
    if (rot) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                S[(size_t)i * n + j] = 0.5 * (Q[(size_t)i * n + j] + Q[(size_t)j * n + i]);
        jacobi_eigen(S, V, n);
        double lmax = 0.0;
        for (int i = 0; i < n; ++i) lmax = std::max(lmax, std::fabs(S[(size_t)i * n + i]));
        for (int i = 0; i < n; ++i) {
            const double l = S[(size_t)i * n + i];
            if (l < -1e-12 * lmax) return *msg = "Q must be positive semidefinite", EMPC_EINVAL;
            o.qd[i] = (float)std::max(l, 0.0);
        }
        // Tm = (A - I) V, then D = V' Tm
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int k = 0; k < n; ++k)
                    s += (A[(size_t)i * n + k] - (i == k ? 1.0 : 0.0)) * V[(size_t)k * n + j];
                Tm[(size_t)i * n + j] = s;
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += V[(size_t)k * n + i] * Tm[(size_t)k * n + j];
                o.D[(size_t)i * n + j] = (float)s;
            }
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += V[(size_t)k * n + i] * B[(size_t)k * m + j];
                o.BT[(size_t)j * n + i] = (float)s;
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) o.Vt[(size_t)i * n + j] = V[(size_t)j * n + i];
    } else {
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j)
                o.D[(size_t)i * n + j] = (float)(A[(size_t)i * n + j] - (i == j ? 1.0 : 0.0));
            for (int j = 0; j < m; ++j) o.BT[(size_t)j * n + i] = (float)B[(size_t)i * m + j];
            o.qd[i] = (float)Q[(size_t)i * n + i];
        }
    }
    for (int i = 0; i < m; ++i) {
        o.rd[i] = (float)R[(size_t)i * m + i];
        if (o.lo) o.lo[i] = (float)bounds[2 * i];
        if (o.hi) o.hi[i] = (float)bounds[2 * i + 1];
    }
    if (dr) {
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double v = 0.5 * (R[(size_t)i * m + j] + R[(size_t)j * m + i]);
                Rs[(size_t)i * m + j] = v;
                o.rmat[(size_t)i * m + j] = (float)v;
            }
        // positive semidefinite: the Jacobi eigenvalues of R_s (S, V reused)
        jacobi_eigen(Rs, S, m);
        double lmax = 0.0;
        for (int i = 0; i < m; ++i) lmax = std::max(lmax, std::fabs(Rs[(size_t)i * m + i]));
        for (int i = 0; i < m; ++i)
            if (Rs[(size_t)i * m + i] < -1e-12 * lmax)
                return *msg = "R must be positive semidefinite", EMPC_EINVAL;
    }
    const long den = T > 1 ? T - 1 : 1;
    for (int k = 0; k < T; ++k) {
        long a = 0, num = 0;
        if (p > 1 && T > 1) {
            a = std::min<long>((long)k * (p - 1) / den, p - 2);
            num = (long)k * (p - 1) - a * den;
        }
        o.idx[k] = (int)a;
        o.w1[k] = (double)num / (double)den;
        o.w0[k] = (double)(den - num) / (double)den;
        o.ks[k].idx1 = (int)a;
        o.ks[k].w0 = (float)o.w0[k];
        o.ks[k].w1 = (float)o.w1[k];
        o.ks[k].pad = 0;
    }
    for (int a = 0; a < p; ++a) Wd[a] = Wo[a] = 0.0;
    for (int k = 0; k < T; ++k) {
        Wd[o.idx[k]] += o.w0[k] * o.w0[k];
        if (p > 1) {
            Wd[o.idx[k] + 1] += o.w1[k] * o.w1[k];
            Wo[o.idx[k]] += o.w0[k] * o.w1[k];
        }
    }
    for (int a = 0; a < p; ++a) {
        o.gram[a] = (float)Wd[a];
        o.gram[p + a] = (float)Wo[a];
    }
    return EMPC_OK;
}

// The tables of one problem in owning vectors (handle and batch APIs).
struct HostTables {
    std::vector<float> D;     // [n][n]  A - I (rollout coordinates)
    std::vector<float> BT;    // [m][n]  B transposed (rollout coordinates)
    std::vector<float> qd;    // [n]     state weights (eigenvalues of Q when rotated)
    std::vector<float> rd;    // [m]     diag(R)
    std::vector<float> lo;    // [m]     u_min
    std::vector<float> hi;    // [m]     u_max
    std::vector<float> gram;  // [2p]    W_aa, W_a,a+1
    std::vector<KnotStep> ks; // [T]
    std::vector<float> rmat;  // [m][m]  symmetric part of R (empty when R is diagonal)
    std::vector<double> Vt;   // [n][n]  x -> z rotation (empty when Q is diagonal)
    std::vector<double> w0, w1;
    std::vector<int> idx;
    bool rotated = false, dense_r = false;

    // z = Vt v in FP64 (the identity when not rotated)
    void rotate(const double* v, double* z, int n) const {
        for (int i = 0; i < n; ++i) {
            if (!rotated) {
                z[i] = v[i];
                continue;
            }
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += Vt[(size_t)i * n + j] * v[j];
            z[i] = s;
        }
    }
};

inline empc_status build_tables(const double* A, const double* B, const double* Q,
                                const double* R, const double* bounds, int n, int m, int T,
                                int p, HostTables& t, std::string& msg) {
    t.D.assign((size_t)n * n, 0.0f);
    t.BT.assign((size_t)m * n, 0.0f);
    t.qd.assign(n, 0.0f);
    t.rd.assign(m, 0.0f);
    t.lo.assign(m, 0.0f);
    t.hi.assign(m, 0.0f);
    t.gram.assign(2 * (size_t)p, 0.0f);
    t.ks.resize(T);
    t.rmat.assign((size_t)m * m, 0.0f);
    t.Vt.assign((size_t)n * n, 0.0);
    t.w0.resize(T);
    t.w1.resize(T);
    t.idx.resize(T);
    std::vector<double> work(table_work_doubles(n, m, p));
    const TableOut o{t.D.data(), t.BT.data(), t.qd.data(), t.rd.data(), t.lo.data(),
                     t.hi.data(), t.gram.data(), t.ks.data(), t.rmat.data(), t.Vt.data(),
                     t.w0.data(), t.w1.data(), t.idx.data(), work.data()};
    const char* m_err = "";
    const empc_status s = fill_tables(A, B, Q, R, bounds, n, m, T, p, o, &t.rotated,
                                      &t.dense_r, &m_err);
    if (s != EMPC_OK) {
        msg = m_err;
        return s;
    }
    if (!t.rotated) t.Vt.clear();
    if (!t.dense_r) t.rmat.clear();
    return EMPC_OK;
}

}  // namespace empc
