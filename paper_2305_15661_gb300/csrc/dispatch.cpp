// Run-time selection of the compiled kernel instantiations.
#include "kernels.h"

namespace ift {

#define IFT_DECL(prob, p, prec) KernelSet kernels_##prob##_##p##_##prec();
#define IFT_DECL_ALL(prob) \
  IFT_DECL(prob, 1, 0) IFT_DECL(prob, 2, 0) IFT_DECL(prob, 3, 0) IFT_DECL(prob, 1, 1) IFT_DECL(prob, 2, 1) \
  IFT_DECL(prob, 3, 1)
IFT_DECL_ALL(1)
IFT_DECL_ALL(2)
IFT_DECL_ALL(3)

static KernelSet pick(int prob, int p, int prec) {
#define IFT_CASE(pr, pp, pc) \
  if (prob == pr && p == pp && prec == pc) return kernels_##pr##_##pp##_##pc();
  IFT_CASE(1, 1, 0) IFT_CASE(1, 2, 0) IFT_CASE(1, 3, 0) IFT_CASE(1, 1, 1) IFT_CASE(1, 2, 1) IFT_CASE(1, 3, 1)
  IFT_CASE(2, 1, 0) IFT_CASE(2, 2, 0) IFT_CASE(2, 3, 0) IFT_CASE(2, 1, 1) IFT_CASE(2, 2, 1) IFT_CASE(2, 3, 1)
  IFT_CASE(3, 1, 0) IFT_CASE(3, 2, 0) IFT_CASE(3, 3, 0) IFT_CASE(3, 1, 1) IFT_CASE(3, 2, 1) IFT_CASE(3, 3, 1)
#undef IFT_CASE
  return KernelSet();
}

KernelSet euler_kernels(int p, int precision) { return pick(2, p, precision); }
KernelSet euler_curved_kernels(int p, int precision) { return pick(3, p, precision); }
KernelSet burgers_kernels(int p, int precision) { return pick(1, p, precision); }

}  // namespace ift
