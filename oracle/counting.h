// Test infrastructure only (see orc.cpp header).
//
// Operation-counting scalar for the oracle's counting build (-DORC_COUNTING).
// It wraps a double and tallies floating-point operations so that the
// algorithmic work per cell-stage can be read off the oracle, which follows
// the paper's steps one by one.  Convention: add/sub/mul count 1, div 1,
// sqrt 1 (counted by the oracle's Sqrt wrapper); negation, fabs, comparisons,
// min and max count 0.  The oracle is compiled with -ffp-contract=off, so
// a*b+c is one mul plus one add (= the 2 flops of an fma).
#pragma once
#include <cmath>

struct OrcCounters {
  unsigned long long add, mul, div, sqrt;
};
// Tallies are kept per phase of the method (see orc.cpp: ORC_PHASE_*).
extern OrcCounters orc_counters[8];
extern int orc_phase;

struct CReal {
  double v;
  CReal() : v(0.0) {}
  CReal(double x) : v(x) {}  // implicit: literals promote
};

inline CReal operator+(CReal a, CReal b) { orc_counters[orc_phase].add++; return CReal(a.v + b.v); }
inline CReal operator-(CReal a, CReal b) { orc_counters[orc_phase].add++; return CReal(a.v - b.v); }
inline CReal operator*(CReal a, CReal b) { orc_counters[orc_phase].mul++; return CReal(a.v * b.v); }
inline CReal operator/(CReal a, CReal b) { orc_counters[orc_phase].div++; return CReal(a.v / b.v); }
inline CReal operator-(CReal a) { return CReal(-a.v); }
inline CReal& operator+=(CReal& a, CReal b) { a = a + b; return a; }
inline CReal& operator-=(CReal& a, CReal b) { a = a - b; return a; }
inline CReal& operator*=(CReal& a, CReal b) { a = a * b; return a; }
inline CReal& operator/=(CReal& a, CReal b) { a = a / b; return a; }
inline bool operator<(CReal a, CReal b) { return a.v < b.v; }
inline bool operator>(CReal a, CReal b) { return a.v > b.v; }
inline bool operator<=(CReal a, CReal b) { return a.v <= b.v; }
inline bool operator>=(CReal a, CReal b) { return a.v >= b.v; }
inline bool operator==(CReal a, CReal b) { return a.v == b.v; }
inline bool operator!=(CReal a, CReal b) { return a.v != b.v; }
