// Shared-memory geometry constants of the FFT stages (host and device).
#pragma once

namespace bem {

// Shared-memory swizzle {a, b, c, d} and row pads (index log2(rows) = 0..6)
// per transform length 2^3 .. 2^13, found by exhaustive search over XOR
// swizzles for conflict-free stage, digit-reversed and split accesses.
struct GeoRow {
  int a, b, c, d, pad[7];
};
constexpr GeoRow kGeo8[11] = {
  {3, 4, 3, 4, {0, 0, 4, 2, 1, 1, 1}},  // L = 8
  {4, 5, 4, 5, {0, 4, 2, 1, 1, 1, 1}},  // L = 16
  {4, 5, 4, 5, {0, 3, 2, 1, 1, 1, 1}},  // L = 32
  {4, 5, 4, 5, {0, 4, 2, 1, 1, 1, 1}},  // L = 64
  {4, 5, 4, 6, {0, 4, 7, 2, 1, 1, 1}},  // L = 128
  {4, 5, 4, 6, {0, 1, 1, 2, 1, 1, 1}},  // L = 256
  {4, 6, 6, 7, {0, 8, 4, 2, 1, 1, 1}},  // L = 512
  {4, 7, 4, 6, {0, 2, 1, 1, 1, 1, 1}},  // L = 1024
  {4, 9, 6, 7, {0, 8, 4, 1, 1, 1, 1}},  // L = 2048
  {4, 9, 4, 6, {0, 8, 1, 1, 1, 1, 1}},  // L = 4096
  {4, 9, 6, 12, {0, 1, 1, 1, 1, 1, 1}},  // L = 8192
};
constexpr GeoRow kGeo16[11] = {
  {3, 4, 3, 4, {0, 4, 2, 1, 1, 1, 1}},  // L = 8
  {3, 4, 3, 4, {0, 2, 2, 1, 1, 1, 1}},  // L = 16
  {3, 4, 3, 4, {0, 4, 2, 1, 1, 1, 1}},  // L = 32
  {3, 4, 3, 6, {0, 4, 2, 1, 1, 1, 1}},  // L = 64
  {3, 5, 3, 4, {0, 4, 2, 1, 1, 1, 1}},  // L = 128
  {3, 5, 3, 7, {0, 1, 2, 1, 1, 1, 1}},  // L = 256
  {3, 6, 5, 8, {0, 4, 2, 1, 1, 1, 1}},  // L = 512
  {3, 6, 5, 9, {0, 2, 1, 1, 1, 1, 1}},  // L = 1024
  {3, 9, 5, 6, {0, 4, 2, 1, 1, 1, 1}},  // L = 2048
  {3, 9, 5, 11, {0, 4, 1, 1, 1, 1, 1}},  // L = 4096
  {3, 9, 5, 12, {0, 1, 1, 1, 1, 1, 1}},  // L = 8192
};


// Compile-time swizzle parameters of a length-2^LOGL transform with ESIZE-byte
// elements (4 = FP32 complex halves, i.e. 8-byte complex; 8 = FP64).
template <int ESIZE, int LOGL>
struct GeoC {
  static constexpr int a = (ESIZE == 4 ? kGeo8 : kGeo16)[LOGL - 3].a;
  static constexpr int b = (ESIZE == 4 ? kGeo8 : kGeo16)[LOGL - 3].b;
  static constexpr int c = (ESIZE == 4 ? kGeo8 : kGeo16)[LOGL - 3].c;
  static constexpr int d = (ESIZE == 4 ? kGeo8 : kGeo16)[LOGL - 3].d;
};

// Swizzles {a, b, c, d} of the radix-16 column transform (lengths 2^9 .. 2^13,
// one column per 2^(LOGL-4) threads, no row pad), same form as above, found by
// exhaustive search for conflict-free stage-0, middle-stage and last-stage
// (digit-reversed group) accesses: 8-byte elements by half-warps, 16-byte
// elements by quarter-warps.
struct GeoR16Row {
  int a, b, c, d;
};
constexpr GeoR16Row kGeoR16_8[5] = {
  {4, 5, 4, 8}, {4, 6, 4, 9}, {4, 7, 4, 10}, {4, 8, 4, 11}, {4, 8, 4, 12}};
constexpr GeoR16Row kGeoR16_16[5] = {
  {3, 4, 3, 8}, {3, 8, 3, 4}, {3, 8, 3, 10}, {3, 8, 3, 10}, {3, 8, 3, 12}};
template <int ESIZE, int LOGL>
struct GeoR16 {
  static constexpr int a = (ESIZE == 4 ? kGeoR16_8 : kGeoR16_16)[LOGL - 9].a;
  static constexpr int b = (ESIZE == 4 ? kGeoR16_8 : kGeoR16_16)[LOGL - 9].b;
  static constexpr int c = (ESIZE == 4 ? kGeoR16_8 : kGeoR16_16)[LOGL - 9].c;
  static constexpr int d = (ESIZE == 4 ? kGeoR16_8 : kGeoR16_16)[LOGL - 9].d;
};

}  // namespace bem
