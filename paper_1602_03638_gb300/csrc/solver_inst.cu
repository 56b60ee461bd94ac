// One (precision, N) instantiation of the solver kernels; compiled once per
// entry of instances.h with DNS_INST_T, DNS_INST_N and DNS_INST_FN defined
// (and DNS_INST_NY, DNS_INST_NZ for a grid with other counts along y and z).
#include "solver_kernels.cuh"

#if !defined(DNS_INST_T) || !defined(DNS_INST_N) || !defined(DNS_INST_FN)
#error "solver_inst.cu needs -DDNS_INST_T=<float|double> -DDNS_INST_N=<N> -DDNS_INST_FN=<name>"
#endif

#ifndef DNS_INST_NY
#define DNS_INST_NY DNS_INST_N
#endif
#ifndef DNS_INST_NZ
#define DNS_INST_NZ DNS_INST_N
#endif

namespace dns {
const DnsOps* DNS_INST_FN() { return SolverImpl<DNS_INST_T, DNS_INST_N, DNS_INST_NY, DNS_INST_NZ>::ops(); }
}  // namespace dns
