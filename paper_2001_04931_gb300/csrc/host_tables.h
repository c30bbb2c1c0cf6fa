// Host-side validation of a problem and construction of the FP32 tables the
// kernels read (shared by the single-problem and batched APIs).
#pragma once
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/empc.h"
#include "empc_internal.h"

namespace empc {

struct HostTables {
    std::vector<float> D;     // [n][n]  A - I
    std::vector<float> BT;    // [m][n]  B transposed
    std::vector<float> qd;    // [n]     diag(Q)
    std::vector<float> rd;    // [m]     diag(R)
    std::vector<float> lo;    // [m]     u_min
    std::vector<float> hi;    // [m]     u_max
    std::vector<float> gram;  // [2p]    W_aa, W_a,a+1
    std::vector<KnotStep> ks; // [T]
    std::vector<double> w0, w1;
    std::vector<int> idx;
};

inline bool all_finite(const double* v, size_t k) {
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Checks the arguments of one problem; returns EMPC_OK or a status with msg.
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
        for (int j = 0; j < n; ++j)
            if (i != j && Q[(size_t)i * n + j] != 0.0)
                return msg = "Q must be diagonal", EMPC_EUNSUPPORTED;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            if (i != j && R[(size_t)i * m + j] != 0.0)
                return msg = "R must be diagonal", EMPC_EUNSUPPORTED;
    for (int i = 0; i < n; ++i)
        if (Q[(size_t)i * n + i] < 0.0) return msg = "Q must be >= 0", EMPC_EINVAL;
    for (int i = 0; i < m; ++i) {
        if (R[(size_t)i * m + i] < 0.0) return msg = "R must be >= 0", EMPC_EINVAL;
        if (!(bounds[2 * i] <= bounds[2 * i + 1])) return msg = "need u_min <= u_max", EMPC_EINVAL;
    }
    return EMPC_OK;
}

// FP32 tables of one problem.  Knot table of Sec. IV-C in exact integers:
// idx1 = min(floor(k (p-1) / (T-1)), p-2), c = (k (p-1) - idx1 (T-1)) / (T-1),
// weights exact rationals rounded once to FP32 (p == 1 or T == 1: constant
// input).  Gram of the weights: sum_k u_k' R u_k = sum_i r_i U_i' W U_i with
// W tridiagonal, W_aa = sum_k w_ka^2, W_a,a+1 = sum_k w_ka w_k,a+1.
inline void build_tables(const double* A, const double* B, const double* Q, const double* R,
                         const double* bounds, int n, int m, int T, int p, HostTables& t) {
    t.D.assign((size_t)n * n, 0.0f);
    t.BT.assign((size_t)m * n, 0.0f);
    t.qd.assign(n, 0.0f);
    t.rd.assign(m, 0.0f);
    t.lo.assign(m, 0.0f);
    t.hi.assign(m, 0.0f);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j)
            t.D[(size_t)i * n + j] = (float)(A[(size_t)i * n + j] - (i == j ? 1.0 : 0.0));
        for (int j = 0; j < m; ++j) t.BT[(size_t)j * n + i] = (float)B[(size_t)i * m + j];
        t.qd[i] = (float)Q[(size_t)i * n + i];
    }
    for (int i = 0; i < m; ++i) {
        t.rd[i] = (float)R[(size_t)i * m + i];
        t.lo[i] = (float)bounds[2 * i];
        t.hi[i] = (float)bounds[2 * i + 1];
    }
    t.ks.resize(T);
    t.w0.resize(T);
    t.w1.resize(T);
    t.idx.resize(T);
    const long den = T > 1 ? T - 1 : 1;
    for (int k = 0; k < T; ++k) {
        long a = 0, num = 0;
        if (p > 1 && T > 1) {
            a = std::min<long>((long)k * (p - 1) / den, p - 2);
            num = (long)k * (p - 1) - a * den;
        }
        t.idx[k] = (int)a;
        t.w1[k] = (double)num / (double)den;
        t.w0[k] = (double)(den - num) / (double)den;
        t.ks[k].idx1 = (int)a;
        t.ks[k].w0 = (float)t.w0[k];
        t.ks[k].w1 = (float)t.w1[k];
        t.ks[k].pad = 0;
    }
    std::vector<double> Wd(p, 0.0), Wo(p, 0.0);
    for (int k = 0; k < T; ++k) {
        Wd[t.idx[k]] += t.w0[k] * t.w0[k];
        if (p > 1) {
            Wd[t.idx[k] + 1] += t.w1[k] * t.w1[k];
            Wo[t.idx[k]] += t.w0[k] * t.w1[k];
        }
    }
    t.gram.assign(2 * (size_t)p, 0.0f);
    for (int a = 0; a < p; ++a) {
        t.gram[a] = (float)Wd[a];
        t.gram[p + a] = (float)Wo[a];
    }
}

}  // namespace empc
