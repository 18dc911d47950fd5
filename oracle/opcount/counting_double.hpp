// A double that counts the floating-point operations done on it (oracle
// op-counting build; test infrastructure only).  +, - and unary minus of a
// difference count as additions, * as multiplications, / as divisions, sqrt
// as square roots; comparisons are counted apart (they are not flops); fabs
// and the conversions are free.
#pragma once
#include <cmath>

struct OpCount { long long add = 0, mul = 0, div = 0, sqrt_ = 0, cmp = 0; };
extern OpCount g_ops;

struct cdouble {
    double v;
    cdouble() : v(0.0) {}
    cdouble(double x) : v(x) {}
    cdouble &operator+=(cdouble o) { g_ops.add++; v += o.v; return *this; }
    cdouble &operator-=(cdouble o) { g_ops.add++; v -= o.v; return *this; }
    cdouble &operator*=(cdouble o) { g_ops.mul++; v *= o.v; return *this; }
    cdouble &operator/=(cdouble o) { g_ops.div++; v /= o.v; return *this; }
    cdouble operator-() const { return cdouble(-v); }
    explicit operator double() const { return v; }
};
inline cdouble operator+(cdouble a, cdouble b) { g_ops.add++; return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { g_ops.add++; return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { g_ops.mul++; return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { g_ops.div++; return cdouble(a.v / b.v); }
inline bool operator<(cdouble a, cdouble b) { g_ops.cmp++; return a.v < b.v; }
inline bool operator>(cdouble a, cdouble b) { g_ops.cmp++; return a.v > b.v; }
inline bool operator<=(cdouble a, cdouble b) { g_ops.cmp++; return a.v <= b.v; }
inline bool operator>=(cdouble a, cdouble b) { g_ops.cmp++; return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { g_ops.cmp++; return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { g_ops.cmp++; return a.v != b.v; }
inline cdouble sqrt(cdouble a) { g_ops.sqrt_++; return cdouble(std::sqrt(a.v)); }
inline cdouble fabs(cdouble a) { return cdouble(std::fabs(a.v)); }
inline cdouble floor(cdouble a) { return cdouble(std::floor(a.v)); }
inline bool isfinite(cdouble a) { return std::isfinite(a.v); }
