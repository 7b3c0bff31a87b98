// FP64 instantiation of the ACM launch wrappers.
#include "acm_ops_impl.cuh"
template struct acm::Ops<double>;
