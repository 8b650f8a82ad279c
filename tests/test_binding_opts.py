"""Host-side marshalling of the assembly options (no GPU): the kernel shape
reaches nl_assemble_opts as 4 doubles, or as NULL for the constant kernel,
and a shape of the wrong length is refused before any call."""
import ctypes as C

import pytest

pytest.importorskip("torch")


def test_constant_kernel_passes_null():
    from paper_2302_07499_gb300 import _binding as B
    o, keep = B._assemble_opts(strategy=B.FULLCAPS, mc_points=32, seed=9, precision=B.FP32_COMP, gamma=2.5)
    assert o.kernel_poly is None
    assert (o.strategy, o.mc_points, o.seed, o.precision, o.gamma) == (B.FULLCAPS, 32, 9, B.FP32_COMP, 2.5)


def test_kernel_shape_passes_its_coefficients():
    from paper_2302_07499_gb300 import _binding as B
    o, keep = B._assemble_opts(kernel=(1.0, -0.6, 0.35, -0.5))
    assert o.kernel_poly
    got = C.cast(o.kernel_poly, C.POINTER(C.c_double))
    assert [got[k] for k in range(4)] == [1.0, -0.6, 0.35, -0.5]


@pytest.mark.parametrize("bad", [(1.0, -1.0, 0.0), (1.0, 0.0, 0.0, 0.0, 0.0)])
def test_kernel_shape_of_wrong_length_is_refused(bad):
    from paper_2302_07499_gb300 import _binding as B
    with pytest.raises(ValueError):
        B._assemble_opts(kernel=bad)


def test_opts_layout_matches_the_header():
    """The ctypes structure lists the fields of nl_assemble_opts in the
    header's order, the kernel shape last."""
    import os
    import re
    from paper_2302_07499_gb300 import _binding as B
    here = os.path.dirname(os.path.abspath(__file__))
    hdr = open(os.path.join(os.path.dirname(here), "include", "nlfem.h")).read()
    body = hdr[:hdr.index("} nl_assemble_opts;")]
    body = body[body.rindex("typedef struct {"):]
    names = re.findall(r"\b(\w+);", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert names == [f for f, _ in B.nl_assemble_opts._fields_]
