// Name -> kernel table of the built-in kernels, and the argument
// introspection call the Python binding uses to marshal values.
#include <string.h>

#include "ecl_internal.h"

namespace ecl {

extern const KernelDesc kMandelbrot;
extern const KernelDesc kGaussian;
extern const KernelDesc kGaussianBatch;
extern const KernelDesc kMandelbrotBatch;
extern const KernelDesc kNBody;
extern const KernelDesc kNBodyAcc;
extern const KernelDesc kNBodyAdjoint;
extern const KernelDesc kNBodyEnergy;
extern const KernelDesc kNBodyFD;
extern const KernelDesc kBinomial;
extern const KernelDesc kBinomialBatch;
extern const KernelDesc kBinomialFull;
extern const KernelDesc kGemmBF16;
extern const KernelDesc kGemmSplit3;
extern const KernelDesc kGemmSplit6;
extern const KernelDesc kCastBF16;
extern const KernelDesc kRay;
extern const KernelDesc kFp32Probe;

static const KernelDesc *const kAll[] = {
    &kMandelbrot,
    &kGaussian,
    &kGaussianBatch,
    &kMandelbrotBatch,
    &kNBody,
    &kNBodyAcc,
    &kNBodyAdjoint,
    &kNBodyEnergy,
    &kNBodyFD,
    &kBinomial,
    &kBinomialBatch,
    &kBinomialFull,
    &kGemmBF16,
    &kGemmSplit3,
    &kGemmSplit6,
    &kCastBF16,
    &kRay,
    &kFp32Probe,
};

const KernelDesc *find_kernel(const char *name)
{
    for (const KernelDesc *k : kAll)
        if (strcmp(k->name, name) == 0) return k;
    return nullptr;
}

}  // namespace ecl

extern "C" ecl_status ecl_kernel_arg(const char *kernel_name, int index, int *kind, const char **name)
{
    const ecl::KernelDesc *k = kernel_name ? ecl::find_kernel(kernel_name) : nullptr;
    if (!k) return ECL_ERR_KERNEL;
    if (index < 0 || index >= k->nargs) return ECL_ERR_ARG;
    if (kind) *kind = (int)k->args[index].kind;
    if (name) *name = k->args[index].name;
    return ECL_OK;
}

extern "C" int ecl_kernel_count(void) { return (int)(sizeof(ecl::kAll) / sizeof(ecl::kAll[0])); }

extern "C" const char *ecl_kernel_name(int i)
{
    if (i < 0 || i >= ecl_kernel_count()) return nullptr;
    return ecl::kAll[i]->name;
}
