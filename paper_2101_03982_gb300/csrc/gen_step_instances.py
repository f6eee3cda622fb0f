"""Write the instantiation files of the fused step, olb_step_<storage>_<D>d.cu.

Each file defines launch_step_<storage>_<D>d and step_info_<storage>_<D>d,
both choosing the kernel from one table, so the launch and its shape always
agree:

* the two-phase kernel (olb_wg.cuh) for p = 3, 4 and the Hermite orders it is
  built for: N = 2, 3 isothermal, N = 4 compressible; the velocity loop is
  unrolled to QM >= Q (9, 27 or 45);
* otherwise the single-role kernel (olb_step.cuh), built for p = 1..6 in FP64
  and p = 2..4 in the shifted storages.

The force_generic argument of launch_step_* and step_info_* is the kernel
mode: 0 automatic, 1 single-role, 2 two-phase (the adjoint's geometry).

FP64 and FP32 files also define launch_adj_<storage>_<D>d, the adjoint step
of the isothermal kernel for p = 3, 4 and the (Q, N) pairs in ADJ_CASES.

Run ``python gen_step_instances.py`` after changing the table.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))

STORAGES = {"f64": "double", "f32": "float", "bf16": "__nv_bfloat16", "f16": "__half"}
GENERIC_P = {"f64": [1, 2, 3, 4, 5, 6], "f32": [2, 3, 4], "bf16": [2, 3, 4], "f16": [2, 3, 4]}
WG_P = [3, 4]
WG_ISO_N = [2, 3]
WG_COMP_N = 4
ADJ_STORAGES = ("f64", "f32")
ADJ_CASES = {2: [(9, 2), (27, 2), (27, 3)], 3: [(27, 2), (27, 3), (45, 2)]}


def iso_qms(D):
    return [9, 27] if D == 2 else [27, 45]


def comp_qm(D):
    return 27 if D == 2 else 45


def wg_cases(D):
    """(P, comp, QM, N) of every two-phase instance of dimension D."""
    out = []
    for P in WG_P:
        for qm in iso_qms(D):
            for N in WG_ISO_N:
                out.append((P, False, qm, N))
        out.append((P, True, comp_qm(D), WG_COMP_N))
    return out


def qm_cond(D, qm, comp):
    if comp:
        return "true"
    qs = iso_qms(D)
    return f"Q <= {qm}" if qm != qs[-1] else "true"


def emit(st, D):
    S = STORAGES[st]
    fn = f"{st}_{D}d"
    L = []
    L.append(f"// Instantiations of the fused step, {S} storage, D = {D}; written by gen_step_instances.py.")
    L.append('#include "olb_wg.cuh"')
    L.append("")
    L.append("namespace olb {")
    L.append("")
    L.append("namespace {")
    L.append(f"using S = {S};")
    L.append("")
    L.append("// Two-phase instance for (P, comp, Q, N): its launch and shape, or null.")
    L.append("using WgLaunch = int (*)(const StepLaunch&);")
    L.append("using WgOcc = int (*)(StepInfo*);")
    L.append("bool pick_wg(int P, int comp, int Q, int N, WgLaunch* l, WgOcc* o) {")
    for (P, comp, qm, N) in wg_cases(D):
        c = "1" if comp else "0"
        targs = f"{D}, {P}, S, {'true' if comp else 'false'}, {qm}, {N}"
        L.append(f"  if (P == {P} && comp == {c} && N == {N} && {qm_cond(D, qm, comp)}) {{")
        L.append(f"    *l = wg::launch_wg<{targs}>;")
        L.append(f"    *o = wg::occupancy_wg<{targs}>;")
        L.append("    return true;")
        L.append("  }")
    L.append("  return false;")
    L.append("}")
    L.append("}  // namespace")
    L.append("")
    L.append(f"int launch_step_{fn}(const StepLaunch& L) {{")
    L.append("  WgLaunch l;")
    L.append("  WgOcc o;")
    L.append("  if (L.force_generic != 1 && pick_wg(L.P, L.compressible, L.a.Q, L.a.N, &l, &o)) return l(L);")
    for P in GENERIC_P[st]:
        for comp in (0, 1):
            L.append(f"  if (L.P == {P} && L.compressible == {comp}) return launch_one<{D}, {P}, S, "
                     f"{'true' if comp else 'false'}>(L);")
    L.append("  return -1;")
    L.append("}")
    L.append("")
    L.append(f"int step_info_{fn}(int P, int comp, int Q, int N, int force_generic, StepInfo* out) {{")
    L.append("  WgLaunch l;")
    L.append("  WgOcc o;")
    L.append("  out->wg = 0;")
    for P in GENERIC_P[st]:
        L.append(f"  if (P == {P}) {{")
        L.append(f"    layout_of<{D}, {P}, S>(out);")
        if P in WG_P:
            L.append("    if (force_generic != 1 && pick_wg(P, comp, Q, N, &l, &o)) {")
            L.append("      out->ctas_per_sm = o(out);  // the two-phase kernel's own tile and shape")
            L.append("      return 0;")
            L.append("    }")
        L.append(f"    out->ctas_per_sm = comp ? occupancy_one<{D}, {P}, S, true>(&out->smem)")
        L.append(f"                            : occupancy_one<{D}, {P}, S, false>(&out->smem);")
        L.append("    return 0;")
        L.append("  }")
    L.append("  return -1;")
    L.append("}")
    L.append("")
    if st in ADJ_STORAGES:
        L.append(f"int launch_adj_{fn}(const StepLaunch& L) {{")
        for P in WG_P:
            for (qm, N) in ADJ_CASES[D]:
                cond = f" && L.a.Q <= {qm}" if qm != iso_qms(D)[-1] else ""
                L.append(f"  if (L.P == {P} && L.a.N == {N}{cond}) return wg::launch_adj<{D}, {P}, S, {qm}, {N}>(L);")
        L.append("  return -1;")
        L.append("}")
        L.append("")
    L.append("}  // namespace olb")
    return "\n".join(L) + "\n"


def main():
    for st in STORAGES:
        for D in (2, 3):
            path = os.path.join(HERE, f"olb_step_{st}_{D}d.cu")
            text = emit(st, D)
            old = open(path).read() if os.path.exists(path) else None
            if old != text:
                with open(path, "w") as f:
                    f.write(text)


if __name__ == "__main__":
    main()
