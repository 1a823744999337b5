"""Write the per-size-class translation units kern_<L>.cu and registry.cu.

    python paper_1305_3699_gb300/csrc/gen_kernels.py

Each size class L (bits) has k channels per base (fixed by the base rule in
setup.cpp), W = L/32 limbs and WX limbs for k*M; every class compiles one or
more lane mappings ("variants": lanes per number TPI, threads per block,
shared-memory vector width).  Variant 0 is the default; others are selected at
run time (mr_set_variant) after measurement.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))

# L: (k, W, WX, [(TPI, THREADS, VEC, MINB[, TC]), ...]).  MINB is the exponentiation kernel's minimum
# resident blocks per SM (its register budget, 0 = compiler's choice), picked per variant by timing
# each value on 1024-16384 numbers of the class with full-length exponents.  TC = 1: the base
# extensions of the exponentiation kernel run on the tensor cores (rns_tc.cuh; 32 numbers per block, 4
# lanes per number in one warp or 8 in two warps; as many blocks per SM as their accumulators fit in
# tensor memory).
CLASSES = {
    512: (18, 16, 17, [(2, 128, 4, 2), (4, 128, 4, 4), (4, 128, 4, 4, 1)]),
    1024: (36, 32, 34, [(4, 128, 4, 2, 1), (4, 128, 4, 3), (8, 128, 4, 4)]),
    1536: (54, 48, 50, [(8, 256, 4, 2, 1), (8, 128, 4, 0)]),
    2048: (72, 64, 66, [(8, 256, 4, 1, 1), (8, 128, 4, 0), (16, 128, 4, 1)]),
    3072: (108, 96, 97, [(16, 256, 4, 0)]),
    4096: (145, 128, 129, [(16, 384, 2, 0)]),
}


# Large classes: several CTAs per group of 32 numbers (big_kernel.cuh).
# L: (k, W, WX, NPT, [(NW, group time relative to variant 0, tensor), ...]).  NW warps per CTA give
# channel slices of 4 NW channels: wider slices need fewer CTAs per group, so more groups fit one
# wave, at a longer time per group (more warps per SM sub-partition).  tensor = 1: the base
# extensions run on the tensor cores (BigTcCfg: 8 warps, 32-channel slices).  The relative group
# times were measured with the variants in one wave on GB300.
BIG = {
    8192: (295, 256, 258, 4, [(8, 1.0, 0), (12, 1.33, 0), (8, 0.495, 1)]),
    16384: (599, 512, 513, 4, [(8, 1.0, 0), (8, 0.434, 1)]),
}


def big_unit(L, k, W, WX, npt, variants):
    out = [f"// Kernel of the {L}-bit size class (k = {k} channels per base). Generated by gen_kernels.py.",
           '#include "big_kernel.cuh"', '#include "kernels_api.h"', "", "namespace mr {", ""]
    entries = []
    for v, (nw, rel, tc) in enumerate(variants):
        C = f"CB{L}v{v}"
        cfg = f"BigTcCfg<{k}, {W}, {WX}>" if tc else f"BigCfg<{k}, {W}, {WX}, {npt}, {nw}>"
        out += [
            f"using {C} = {cfg};",
            f"static size_t slot_words_{L}_{v}(uint32_t wbits) {{ return {C}::slot_words(wbits); }}", "",
            f"static cudaError_t launch_big_{L}_{v}(const BigArgs& a, cudaStream_t s) {{",
            "  void* args[] = {const_cast<BigArgs*>(&a)};",
            f"  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<{C}>, dim3(a.slots * {C}::SLICES),",
            f"                                     dim3({C}::THREADS), args, {C}::SMEM_BYTES, s);", "}", "",
            f"static cudaError_t prepare_big_{L}_{v}() {{",
            f"  return cudaFuncSetAttribute(big_modexp_kernel<{C}>, cudaFuncAttributeMaxDynamicSharedMemorySize, {C}::SMEM_BYTES);",
            "}", "",
            f"static int occupancy_big_{L}_{v}() {{",
            "  int n = 0;",
            f"  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<{C}>, {C}::THREADS, {C}::SMEM_BYTES) != cudaSuccess) n = 0;",
            "  return n;", "}", ""]
        entries.append(f"    {{{C}::SC, {C}::SLICES, {C}::THREADS, {C}::SMEM_BYTES, {tc}, {rel:.3f}f, slot_words_{L}_{v}, "
                       f"launch_big_{L}_{v}, prepare_big_{L}_{v}, occupancy_big_{L}_{v}}}")
    out.append(f"static const BigKernel kBig{L}[{len(variants)}] = {{")
    out.append(",\n".join(entries) + "};")
    out.append(f"extern const ClassKernels kClass{L} = {{{L}, {k}, {W}, {WX}, 0, {{}}, kBig{L}, {len(variants)}}};")
    out += ["", "}  // namespace mr", ""]
    return "\n".join(out)


def unit(L, k, W, WX, variants):
    out = [f"// Kernels of the {L}-bit size class (k = {k} channels per base). Generated by gen_kernels.py.",
           '#include "kernels.cuh"', '#include "kernels_api.h"', '#include "mr_kernel.cuh"', "", "namespace mr {", ""]
    entries = []
    for v, var in enumerate(variants):
        tpi, th, vec, minb = var[:4]
        tc = var[4] if len(var) > 4 else 0
        C = f"C{L}v{v}"
        out.append(f"using {C} = Cfg<{k}, {W}, {WX}, {tpi}, {th}, {vec}, {minb}, {tc}>;")
        for kind, kern, argt, sm in (("modexp", "modexp_kernel", "LaunchArgs", "SMEM_MODEXP_BYTES"),
                                     ("crt", "crt_kernel", "LaunchArgs", "SMEM_BYTES"),
                                     ("mr", "mr_kernel", "MRArgs", "SMEM_BYTES")):
            out += [f"static cudaError_t launch_{kind}_{L}_{v}(const {argt}& a, unsigned grid, cudaStream_t s) {{",
                    f"  {kern}<{C}><<<grid, {C}::THREADS, {C}::{sm}, s>>>(a);",
                    "  return cudaGetLastError();", "}", ""]
        out += [f"static cudaError_t prepare_{L}_{v}() {{",
                "  cudaError_t e = cudaSuccess, r;",
                f"  if ((r = cudaFuncSetAttribute(modexp_kernel<{C}>, cudaFuncAttributeMaxDynamicSharedMemorySize, {C}::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;",
                f"  if ((r = cudaFuncSetAttribute(crt_kernel<{C}>, cudaFuncAttributeMaxDynamicSharedMemorySize, {C}::SMEM_BYTES)) != cudaSuccess) e = r;",
                f"  if ((r = cudaFuncSetAttribute(mr_kernel<{C}>, cudaFuncAttributeMaxDynamicSharedMemorySize, {C}::SMEM_BYTES)) != cudaSuccess) e = r;",
                "  return e;", "}", "",
                f"static int occupancy_{L}_{v}() {{",
                "  int n = 0;",
                f"  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<{C}>, {C}::THREADS, {C}::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;",
                "  return n > 0 ? n : 1;", "}", ""]
        entries.append(f"     {{{C}::TPI, {C}::THREADS, {C}::IPB, {C}::NPT, {C}::SMEM_MODEXP_BYTES, {C}::TC, launch_modexp_{L}_{v}, "
                       f"launch_crt_{L}_{v}, launch_mr_{L}_{v}, prepare_{L}_{v}, occupancy_{L}_{v}}}")
    out.append(f"extern const ClassKernels kClass{L} = {{")
    out.append(f"    {L}, {k}, {W}, {WX}, {len(variants)},")
    out.append("    {\n" + ",\n".join(entries) + "},")
    out.append("    nullptr, 0};")
    out += ["", "}  // namespace mr", ""]
    return "\n".join(out)


def main():
    for L, (k, W, WX, vs) in CLASSES.items():
        with open(os.path.join(HERE, f"kern_{L}.cu"), "w") as f:
            f.write(unit(L, k, W, WX, vs))
    for L, (k, W, WX, npt, vs) in BIG.items():
        with open(os.path.join(HERE, f"kern_{L}.cu"), "w") as f:
            f.write(big_unit(L, k, W, WX, npt, vs))
    allc = list(CLASSES) + list(BIG)
    reg = ["// Registry of the compiled size classes. Generated by gen_kernels.py.", '#include "kernels_api.h"', "",
           "namespace mr {", ""]
    reg += [f"extern const ClassKernels kClass{L};" for L in allc]
    reg += ["", "const ClassKernels* class_kernels(uint32_t L) {", "  switch (L) {"]
    for L in allc:
        reg += [f"    case {L}:", f"      return &kClass{L};"]
    reg += ["    default:", "      return nullptr;", "  }", "}", "", "}  // namespace mr", ""]
    with open(os.path.join(HERE, "registry.cu"), "w") as f:
        f.write("\n".join(reg))


if __name__ == "__main__":
    main()
