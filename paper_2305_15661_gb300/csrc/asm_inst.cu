// One instantiation of the element kernels, selected at compile time by
// IFT_PROB (1 Burgers, 2 Euler, 3 Euler on curved elements), IFT_P (degree) and
// IFT_PREC (0 FP64, 1 FP32).
// The build compiles this file once per combination, in parallel.
#include "kernel_set.cuh"

#if !defined(IFT_PROB) || !defined(IFT_P) || !defined(IFT_PREC)
#error "IFT_PROB, IFT_P and IFT_PREC must be defined"
#endif

#define IFT_CAT_(a, b, c, d) a##_##b##_##c##_##d
#define IFT_CAT(a, b, c, d) IFT_CAT_(a, b, c, d)

namespace ift {

KernelSet IFT_CAT(kernels, IFT_PROB, IFT_P, IFT_PREC)() {
#if IFT_PREC == 0
  return KernelSetImpl<double, IFT_PROB, IFT_P>::make();
#else
  return KernelSetImpl<float, IFT_PROB, IFT_P>::make();
#endif
}

}  // namespace ift
