// Operation tally of the FP64 oracle (test infrastructure only, like the rest
// of oracle/): the oracle's C source compiled with every `double` replaced by
// a scalar type that counts its arithmetic.  The values it computes are the
// oracle's own (the type wraps one double and rounds like it); only the
// counts are new.  Used to state the method's operations per cell-stage, not
// to check results.
//
// Counted: additions, subtractions, multiplications and divisions with at
// least one non-constant operand, each as one floating-point operation;
// square roots, exponentials, erfc and powers as special functions.
// Comparisons, fabs and copies are free.  A second tally leaves out the
// operations whose result needs no arithmetic: an addition or subtraction of
// an exact zero, a multiplication by an exact zero or +-1, a division by +-1
// (the generic moment expansions of the oracle multiply by many structural
// zeros and ones).
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace fc {
struct Tally {
    unsigned long long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, erfc = 0, pow = 0;
    unsigned long long add_nt = 0, mul_nt = 0, div_nt = 0;  // non-trivial operands only
};
static Tally tally;

inline bool unit(double x) { return x == 1.0 || x == -1.0; }
inline void t_add(double a, double b) { ++tally.add; if (a != 0.0 && b != 0.0) ++tally.add_nt; }
inline void t_mul(double a, double b)
{
    ++tally.mul;
    if (a != 0.0 && b != 0.0 && !unit(a) && !unit(b)) ++tally.mul_nt;
}
inline void t_div(double a, double b) { ++tally.div; if (a != 0.0 && !unit(b)) ++tally.div_nt; }

struct cd {
    double v;
    cd() = default;
    cd(double x) : v(x) {}
    cd& operator+=(cd o) { t_add(v, o.v); v += o.v; return *this; }
    cd& operator-=(cd o) { t_add(v, o.v); v -= o.v; return *this; }
    cd& operator*=(cd o) { t_mul(v, o.v); v *= o.v; return *this; }
    cd& operator/=(cd o) { t_div(v, o.v); v /= o.v; return *this; }
    cd operator-() const { return cd(-v); }
    explicit operator int() const { return (int)v; }
};
inline cd operator+(cd a, cd b) { t_add(a.v, b.v); return cd(a.v + b.v); }
inline cd operator-(cd a, cd b) { t_add(a.v, b.v); return cd(a.v - b.v); }
inline cd operator*(cd a, cd b) { t_mul(a.v, b.v); return cd(a.v * b.v); }
inline cd operator/(cd a, cd b) { t_div(a.v, b.v); return cd(a.v / b.v); }
inline bool operator<(cd a, cd b) { return a.v < b.v; }
inline bool operator>(cd a, cd b) { return a.v > b.v; }
inline bool operator<=(cd a, cd b) { return a.v <= b.v; }
inline bool operator>=(cd a, cd b) { return a.v >= b.v; }
inline bool operator==(cd a, cd b) { return a.v == b.v; }
inline bool operator!=(cd a, cd b) { return a.v != b.v; }
inline cd fabs(cd a) { return cd(std::fabs(a.v)); }
inline cd sqrt(cd a) { ++tally.sqrt; return cd(std::sqrt(a.v)); }
inline cd exp(cd a) { ++tally.exp; return cd(std::exp(a.v)); }
inline cd erfc(cd a) { ++tally.erfc; return cd(std::erfc(a.v)); }
inline cd pow(cd a, int n) { ++tally.pow; return cd(std::pow(a.v, n)); }
inline cd pow(cd a, cd b) { ++tally.pow; return cd(std::pow(a.v, b.v)); }
inline bool isfinite(cd a) { return std::isfinite(a.v); }
}  // namespace fc

using fc::cd;
using std::erfc;
using std::exp;
using std::fabs;
using std::isfinite;
using std::pow;
using std::sqrt;

#define double cd
extern "C" {
#include "cgks_oracle.c"
}
#undef double

extern "C" void oracle_tally_reset(void) { fc::tally = fc::Tally(); }

// [add, mul, div, sqrt, exp, erfc, pow, add_nt, mul_nt, div_nt]
extern "C" void oracle_tally_get(unsigned long long* out)
{
    out[0] = fc::tally.add; out[1] = fc::tally.mul; out[2] = fc::tally.div;
    out[3] = fc::tally.sqrt; out[4] = fc::tally.exp; out[5] = fc::tally.erfc; out[6] = fc::tally.pow;
    out[7] = fc::tally.add_nt; out[8] = fc::tally.mul_nt; out[9] = fc::tally.div_nt;
}
