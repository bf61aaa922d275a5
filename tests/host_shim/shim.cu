// Test shim: the library's __host__ __device__ primitives compiled for the
// host, so the CPU test-suite can compare their arithmetic with the oracle
// before any GPU run.  Not part of the library.
#include "kg_common.cuh"

using namespace kg;

extern "C" {
double sh_log(double x) { return kg_log(x); }
double sh_log1m(double p) { return kg_log1m(p); }
double sh_exp(double x) { return kg_exp(x); }
double sh_lnfact(double k) { return kg_lnfact(k); }
double sh_lnfact_diff(double a, double d) { return kg_lnfact_diff(a, d); }
double sh_dbl128(uint64_t lo, uint64_t hi) { return dbl((u128(hi) << 64) | lo); }
uint64_t sh_stream_u64(uint64_t seed, uint64_t node, uint32_t tag, uint64_t i) {
  return stream_u64(seed, node, tag, i);
}
int sh_hyper(uint64_t Nlo, uint64_t Nhi, uint64_t Klo, uint64_t Khi, uint64_t t, uint64_t seed,
             uint64_t node, uint32_t tag, uint64_t* x) {
  Stream s(seed, node, tag);
  return hypergeometric((u128(Nhi) << 64) | Nlo, (u128(Khi) << 64) | Klo, t, s, *x);
}
int sh_binom(uint64_t n, double p, uint64_t seed, uint64_t node, uint32_t tag, uint64_t* x) {
  Stream s(seed, node, tag);
  return binomial(n, p, s, *x);
}
uint64_t sh_lemire(uint64_t seed, uint64_t node, uint64_t i, uint64_t range) {
  return lemire_draw(stream_u64(seed, node, TAG_LEAF, i), range, seed, node, i);
}
// floor(x / D) through the invariant-division multiplier, for a batch
void sh_divq(uint64_t D, const uint64_t* x, uint64_t* q, uint64_t count) {
  const DivU64 d = make_div(D);
  for (uint64_t i = 0; i < count; ++i) q[i] = div_q(d, x[i]);
}
void sh_und_map(uint64_t n, uint32_t P, uint64_t k, uint64_t off, uint64_t* u, uint64_t* v) {
  UndGeom g{n, P, RowBounds::make(n, P)};
  g.map(g.ctx(k), off, *u, *v);
}
uint64_t sh_und_universe(uint64_t n, uint32_t P, uint64_t k) {
  UndGeom g{n, P, RowBounds::make(n, P)};
  return g.universe(k);
}
uint64_t sh_row_bound(uint64_t n, uint32_t P, uint64_t c) { return RowBounds::make(n, P)(c); }
}
