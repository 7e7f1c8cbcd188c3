/* opcount.h -- the oracle's floating-point operation counter (test infrastructure only).
 *
 * Included by npxo.c only when it is compiled as C++ with NPXO_OPCOUNT defined (oracle.py builds
 * that as a second library, libnpxo_count.so, from the same source).  Every `double` of the
 * oracle then becomes npxo_cdouble: a wrapper holding one double that performs exactly the same
 * IEEE operations in the same order (so the counting build steps bit-identically to the plain
 * one) and counts each of them into the region the oracle is executing (NPXO_REGION in npxo.c):
 * additions and subtractions, multiplications, divisions, square roots, calls of sin / cos /
 * asin, and comparisons.  Negation, fabs and copies are not counted.  The counts are global and
 * not thread-safe: the counting build is stepped on one thread.
 */
#ifndef NPXO_OPCOUNT_H
#define NPXO_OPCOUNT_H
#ifndef __cplusplus
#error "opcount.h is for the C++ counting build of the oracle"
#endif
#include <math.h>

enum { NPXO_R_OTHER = 0, NPXO_R_SCENE, NPXO_R_POINT, NPXO_R_CONTACT, NPXO_R_FRICTION, NPXO_R_TICK,
       NPXO_R_N };
enum { NPXO_K_ADD = 0, NPXO_K_MUL, NPXO_K_DIV, NPXO_K_SQRT, NPXO_K_TRANSC, NPXO_K_CMP, NPXO_K_N };

extern unsigned long long npxo_ops[NPXO_R_N][NPXO_K_N];
extern int npxo_region;

#define NPXO_REGION(r) (npxo_region = (r))
#define NPXO_COUNT(kind, n) (npxo_ops[npxo_region][kind] += (n))

struct npxo_cdouble {
    double v;
    npxo_cdouble() = default;
    npxo_cdouble(double x) : v(x) {}
    explicit operator float() const { return (float)v; }
    explicit operator double() const { return v; }
    explicit operator long long() const { return (long long)v; }
    explicit operator int() const { return (int)v; }
    npxo_cdouble operator-() const { return npxo_cdouble(-v); }
    npxo_cdouble &operator+=(npxo_cdouble o) { NPXO_COUNT(NPXO_K_ADD, 1); v += o.v; return *this; }
    npxo_cdouble &operator-=(npxo_cdouble o) { NPXO_COUNT(NPXO_K_ADD, 1); v -= o.v; return *this; }
    npxo_cdouble &operator*=(npxo_cdouble o) { NPXO_COUNT(NPXO_K_MUL, 1); v *= o.v; return *this; }
    npxo_cdouble &operator/=(npxo_cdouble o) { NPXO_COUNT(NPXO_K_DIV, 1); v /= o.v; return *this; }
};
typedef npxo_cdouble cd_;
inline cd_ operator+(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_ADD, 1); return cd_(a.v + b.v); }
inline cd_ operator-(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_ADD, 1); return cd_(a.v - b.v); }
inline cd_ operator*(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_MUL, 1); return cd_(a.v * b.v); }
inline cd_ operator/(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_DIV, 1); return cd_(a.v / b.v); }
inline bool operator<(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v < b.v; }
inline bool operator>(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v > b.v; }
inline bool operator<=(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v <= b.v; }
inline bool operator>=(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v >= b.v; }
inline bool operator==(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v == b.v; }
inline bool operator!=(cd_ a, cd_ b) { NPXO_COUNT(NPXO_K_CMP, 1); return a.v != b.v; }
inline cd_ sqrt(cd_ a) { NPXO_COUNT(NPXO_K_SQRT, 1); return cd_(::sqrt(a.v)); }
inline cd_ sin(cd_ a) { NPXO_COUNT(NPXO_K_TRANSC, 1); return cd_(::sin(a.v)); }
inline cd_ cos(cd_ a) { NPXO_COUNT(NPXO_K_TRANSC, 1); return cd_(::cos(a.v)); }
inline cd_ asin(cd_ a) { NPXO_COUNT(NPXO_K_TRANSC, 1); return cd_(::asin(a.v)); }
inline cd_ fabs(cd_ a) { return cd_(::fabs(a.v)); }
inline bool isfinite(cd_ a) { return std::isfinite(a.v); }
inline long long llround(cd_ a) { return ::llround(a.v); }

/* from here on the oracle's doubles count */
#define double npxo_cdouble
#endif
