/*
 * Operation-counting build of the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * oracle/__init__.py compiles mfc_oracle.c a second time, as C++ with this
 * header forced in front of it and `double` redefined to `fc_real`, a
 * one-member struct with the size, alignment and values of a double whose
 * arithmetic operators bump a counter.  The oracle's source is unchanged, so
 * the count is that of the plain textbook formulation (the paper's algorithmic
 * work), independent of how the CUDA kernels fold or fuse it.
 *
 * Counted, one each: + - * / (binary, compound forms included) and sqrt.
 * Not counted: comparisons, unary minus, fabs, fmin, fmax, isfinite, isnan,
 * conversions.  Single-threaded (no OpenMP), so one global counter suffices.
 */
#ifndef ORACLE_FLOP_COUNT_H
#define ORACLE_FLOP_COUNT_H

/* the system headers first, with the real double */
#include <math.h>
#include <cmath>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

extern "C" {
unsigned long long oracle_flop_counter = 0;
void oracle_flop_reset(void) { oracle_flop_counter = 0; }
unsigned long long oracle_flop_read(void) { return oracle_flop_counter; }
}

struct fc_real {
    double v;
    fc_real() = default;
    constexpr fc_real(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    fc_real& operator+=(fc_real o) { ++oracle_flop_counter; v += o.v; return *this; }
    fc_real& operator-=(fc_real o) { ++oracle_flop_counter; v -= o.v; return *this; }
    fc_real& operator*=(fc_real o) { ++oracle_flop_counter; v *= o.v; return *this; }
    fc_real& operator/=(fc_real o) { ++oracle_flop_counter; v /= o.v; return *this; }
};
static_assert(sizeof(fc_real) == sizeof(double) && alignof(fc_real) == alignof(double), "layout of double");

static inline fc_real operator+(fc_real a, fc_real b) { ++oracle_flop_counter; return fc_real(a.v + b.v); }
static inline fc_real operator-(fc_real a, fc_real b) { ++oracle_flop_counter; return fc_real(a.v - b.v); }
static inline fc_real operator*(fc_real a, fc_real b) { ++oracle_flop_counter; return fc_real(a.v * b.v); }
static inline fc_real operator/(fc_real a, fc_real b) { ++oracle_flop_counter; return fc_real(a.v / b.v); }
static inline fc_real operator-(fc_real a) { return fc_real(-a.v); }
static inline fc_real operator+(fc_real a) { return a; }
static inline bool operator<(fc_real a, fc_real b) { return a.v < b.v; }
static inline bool operator<=(fc_real a, fc_real b) { return a.v <= b.v; }
static inline bool operator>(fc_real a, fc_real b) { return a.v > b.v; }
static inline bool operator>=(fc_real a, fc_real b) { return a.v >= b.v; }
static inline bool operator==(fc_real a, fc_real b) { return a.v == b.v; }
static inline bool operator!=(fc_real a, fc_real b) { return a.v != b.v; }
static inline fc_real sqrt(fc_real a) { ++oracle_flop_counter; return fc_real(std::sqrt(a.v)); }
static inline fc_real fabs(fc_real a) { return fc_real(std::fabs(a.v)); }
static inline fc_real fmin(fc_real a, fc_real b) { return fc_real(std::fmin(a.v, b.v)); }
static inline fc_real fmax(fc_real a, fc_real b) { return fc_real(std::fmax(a.v, b.v)); }
static inline bool isfinite(fc_real a) { return std::isfinite(a.v); }
static inline bool isnan(fc_real a) { return std::isnan(a.v); }

#define double fc_real
#endif
