// flopcount.cpp -- operation counts of the oracle's step: the algorithmic
// work of the method, per cell-update and per stage.
//
// TEST AND MEASUREMENT INFRASTRUCTURE ONLY (like the oracle itself): only the
// tests and the benchmark's roofline numerator use it.
//
// The oracle's own source (mhd_oracle.c) is compiled here unchanged, as C++,
// with its floating-point type replaced by `fc_real`: a double that counts every
// addition/subtraction, multiplication, division, square root, comparison
// (min, max, branch tests) and absolute value it performs.  Integer index
// arithmetic is not counted.  The oracle's stage marks (ORC_STAGE) attribute
// the operations since the previous mark to a named stage.  Built without
// OpenMP (single-threaded, so the counters are exact).
//
// Build: g++ -O1 -std=c++17 -ffp-contract=off -shared -fPIC flopcount.cpp
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <string>
#include <type_traits>

namespace fc {
struct Counts {
    long long add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0, abs = 0;
    long long add0 = 0, mul0 = 0;   // of add, mul: with an operand that is exactly 0 (or a factor +-1)
};
static Counts total;
static std::map<std::string, Counts> stages;
static Counts at_mark;

static void mark(const char* name)
{
    Counts& s = stages[name];
    s.add += total.add - at_mark.add;
    s.mul += total.mul - at_mark.mul;
    s.div += total.div - at_mark.div;
    s.sqrt += total.sqrt - at_mark.sqrt;
    s.cmp += total.cmp - at_mark.cmp;
    s.abs += total.abs - at_mark.abs;
    s.add0 += total.add0 - at_mark.add0;
    s.mul0 += total.mul0 - at_mark.mul0;
    at_mark = total;
}
// an addition with a zero operand, or a multiplication by 0 or +-1, is
// counted and also tallied as trivial: the plain oracle multiplies whole
// eigenvector matrices, whose structural zeros a dense count would include
static inline void count_add(double a, double b)
{
    total.add++;
    if (a == 0.0 || b == 0.0) total.add0++;
}
static inline void count_mul(double a, double b)
{
    total.mul++;
    if (a == 0.0 || b == 0.0 || a == 1.0 || b == 1.0 || a == -1.0 || b == -1.0) total.mul0++;
}
}  // namespace fc

// a double that counts its floating-point operations; same size and layout
// as double, so the oracle's arrays are passed in unchanged
struct fc_real {
    double v;
    fc_real() = default;
    template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
    fc_real(T x) : v((double)x) {}
    explicit operator double() const { return v; }
    fc_real& operator+=(fc_real o) { fc::count_add(v, o.v); v += o.v; return *this; }
    fc_real& operator-=(fc_real o) { fc::count_add(v, o.v); v -= o.v; return *this; }
    fc_real& operator*=(fc_real o) { fc::count_mul(v, o.v); v *= o.v; return *this; }
    fc_real& operator/=(fc_real o) { fc::total.div++; v /= o.v; return *this; }
};
static_assert(sizeof(fc_real) == sizeof(double), "fc_real must alias double");

static inline fc_real operator+(fc_real a, fc_real b) { fc::count_add(a.v, b.v); return fc_real(a.v + b.v); }
static inline fc_real operator-(fc_real a, fc_real b) { fc::count_add(a.v, b.v); return fc_real(a.v - b.v); }
static inline fc_real operator*(fc_real a, fc_real b) { fc::count_mul(a.v, b.v); return fc_real(a.v * b.v); }
static inline fc_real operator/(fc_real a, fc_real b) { fc::total.div++; return fc_real(a.v / b.v); }
static inline fc_real operator-(fc_real a) { return fc_real(-a.v); }            // a sign flip, not counted
static inline fc_real operator+(fc_real a) { return a; }
static inline bool operator<(fc_real a, fc_real b) { fc::total.cmp++; return a.v < b.v; }
static inline bool operator>(fc_real a, fc_real b) { fc::total.cmp++; return a.v > b.v; }
static inline bool operator<=(fc_real a, fc_real b) { fc::total.cmp++; return a.v <= b.v; }
static inline bool operator>=(fc_real a, fc_real b) { fc::total.cmp++; return a.v >= b.v; }
static inline bool operator==(fc_real a, fc_real b) { fc::total.cmp++; return a.v == b.v; }
static inline bool operator!=(fc_real a, fc_real b) { fc::total.cmp++; return a.v != b.v; }
static inline fc_real sqrt(fc_real a) { fc::total.sqrt++; return fc_real(std::sqrt(a.v)); }
static inline fc_real fabs(fc_real a) { fc::total.abs++; return fc_real(std::fabs(a.v)); }

#define ORC_STAGE(name) fc::mark(name)
#define double fc_real
extern "C" {
#include "mhd_oracle.c"
}
#undef double

extern "C" {

// Clear every counter.
void fc_reset(void)
{
    fc::total = fc::Counts();
    fc::at_mark = fc::Counts();
    fc::stages.clear();
}

// Attribute the operations since the last mark to `name` (e.g. "cfl").
void fc_mark(const char* name) { fc::mark(name); }

// Totals: out[8] = add, mul, div, sqrt, cmp, abs, trivial add, trivial mul.
void fc_totals(long long* out)
{
    const fc::Counts& c = fc::total;
    out[0] = c.add; out[1] = c.mul; out[2] = c.div; out[3] = c.sqrt; out[4] = c.cmp; out[5] = c.abs;
    out[6] = c.add0; out[7] = c.mul0;
}

// Number of stages recorded, and the i-th (name into buf, counts into out[8]).
int fc_nstages(void) { return (int)fc::stages.size(); }
void fc_stage(int i, char* buf, int buflen, long long* out)
{
    auto it = fc::stages.begin();
    std::advance(it, i);
    std::strncpy(buf, it->first.c_str(), (size_t)buflen - 1);
    buf[buflen - 1] = 0;
    const fc::Counts& c = it->second;
    out[0] = c.add; out[1] = c.mul; out[2] = c.div; out[3] = c.sqrt; out[4] = c.cmp; out[5] = c.abs;
    out[6] = c.add0; out[7] = c.mul0;
}

}  // extern "C"
