// Length limit of the correctly rounded dot product (exact_dot.cuh), shared
// by every entry point that runs it.
#pragma once

namespace airg {

// Each 64-bit digit of the fixed-point accumulator receives at most one
// 32-bit piece per product, so fewer than 2^31 products cannot carry out of
// a digit.
constexpr long long XD_MAX_N = (1LL << 31) - 1;

}  // namespace airg
