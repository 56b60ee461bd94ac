// Grid sizes and precisions compiled into the library. Each entry X(T, tag, N)
// becomes one translation unit (solver_inst.cu built with -DDNS_INST_T=T
// -DDNS_INST_N=N -DDNS_INST_FN=dns_ops_<tag>_<N>); each entry
// B(T, tag, NX, NY, NZ) of DNS_BOX_INSTANCES one more for a grid with other
// point counts per direction (-DDNS_INST_NY, -DDNS_INST_NZ,
// -DDNS_INST_FN=dns_ops_<tag>_<NX>x<NY>x<NZ>).
#pragma once

#define DNS_INSTANCES(X)                                                                          \
  X(float, f32, 8) X(float, f32, 12) X(float, f32, 16) X(float, f32, 24) X(float, f32, 32)        \
  X(float, f32, 48) X(float, f32, 64) X(float, f32, 96) X(float, f32, 128) X(float, f32, 256)    \
  X(float, f32, 512) X(float, f32, 1024)                                                          \
  X(double, f64, 8) X(double, f64, 12) X(double, f64, 16) X(double, f64, 24) X(double, f64, 32)  \
  X(double, f64, 48) X(double, f64, 64) X(double, f64, 96) X(double, f64, 128)                   \
  X(double, f64, 256) X(double, f64, 512) X(double, f64, 1024)

// Grids with a different number of points per direction (generic passes only):
// small ones for the parity tests, 1024 x 512 x 256 for measurement.
#define DNS_BOX_INSTANCES(B)                                                                      \
  B(float, f32, 32, 16, 24) B(double, f64, 32, 16, 24) B(float, f32, 24, 48, 16)                 \
  B(double, f64, 24, 48, 16) B(float, f32, 1024, 512, 256) B(double, f64, 1024, 512, 256)
