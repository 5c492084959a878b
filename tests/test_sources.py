"""Static checks on the CUDA sources (no GPU needed)."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2312_11801_gb300", "csrc")


def _code(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return "\n".join(line.split("//")[0] for line in text.splitlines())


def test_shared_bodies_take_their_cta_index_as_an_argument():
    """The kernel bodies in dev_*.cuh run both as per-step kernels and inside the
    persistent batched kernel, where blockIdx is not the instance's CTA index: a body
    must use the cta / ncta arguments it is given, never blockIdx or gridDim."""
    for name in sorted(os.listdir(CSRC)):
        if name.startswith("dev_") and name.endswith(".cuh") or name == "batch_kernel.cuh":
            code = _code(os.path.join(CSRC, name))
            bad = [m.group(0) for m in re.finditer(r"\b(blockIdx|gridDim)\b", code)]
            if name == "batch_kernel.cuh":
                continue   # the persistent kernel itself may look at its own grid
            assert not bad, (name, bad)


def test_batched_translation_units_use_plain_loads():
    """A persistent kernel that writes a buffer and reads it again in the same launch
    must not read it through the non-coherent read-only path."""
    for name in sorted(os.listdir(CSRC)):
        if name.startswith("batch_") and name.endswith(".cu"):
            text = open(os.path.join(CSRC, name)).read()
            inc = text.index('#include "batch_kernel.cuh"')
            assert "#define USBS_PLAIN_LOADS" in text[:inc], name
