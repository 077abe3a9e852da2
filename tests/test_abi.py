"""The C ABI library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here (no GPU on the build host)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "helm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1502_07266_gb300.helm import _LIB_PATH
    return _LIB_PATH


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("helm_setup", "helm_apply_precond", "helm_solve", "helm_matvec",
                     "helm_destroy", "helm_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1502_07266_gb300 import helm
    assert set(_declared_functions()) == set(helm.EXPORTED)


def test_host_only_calls(libpath):
    """Calls that touch no device: defaults, error strings, argument checks."""
    from paper_1502_07266_gb300 import helm
    o = helm.helm_default_opts()
    assert (o.restart, o.maxit, o.pml_C, o.b_aux) == (30, 300, 10.0, 0)
    assert "invalid" in helm.helm_strerror(helm.HELM_EINVAL)
    L = helm.lib()
    h = ctypes.c_void_p()
    # null velocity pointer and bad sizes are rejected before any CUDA call
    assert L.helm_setup(None, 1.0, 7, 3, 1, None, None, ctypes.byref(h)) == helm.HELM_EINVAL
    assert L.helm_setup(ctypes.c_void_p(16), 1.0, 0, 3, 1, None, None, ctypes.byref(h)) == helm.HELM_EINVAL
    assert L.helm_setup(ctypes.c_void_p(16), -1.0, 7, 3, 1, None, None, ctypes.byref(h)) == helm.HELM_EINVAL
    assert L.helm_apply_precond(None, None, None, 1, None) == helm.HELM_EINVAL
    assert L.helm_solve(None, None, None, 1, 1e-6, None, None, None) == helm.HELM_EINVAL
    # options are validated before any device work
    bad = helm.helm_default_opts()
    bad.apply_form = 7
    assert L.helm_setup(ctypes.c_void_p(16), 1.0, 7, 3, 1, ctypes.byref(bad), None, ctypes.byref(h)) == helm.HELM_EINVAL
    bad = helm.helm_default_opts()
    bad.wait_cycles = -1
    assert L.helm_setup(ctypes.c_void_p(16), 1.0, 7, 3, 1, ctypes.byref(bad), None, ctypes.byref(h)) == helm.HELM_EINVAL
    assert L.helm_dense_operator(None, 0, 0, 0, None, None, None, None, None) == helm.HELM_ENOTSUP
    L.helm_destroy(None)


def test_product_path_does_not_import_the_oracle():
    """The binding and the CUDA sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1502_07266_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(^|\n)\s*(from|import)\s+oracle\b", src), f
                assert "oracle/" not in src and "oracle." not in src, f


def test_pad_velocity_is_the_nearest_value_extension():
    """pad_velocity extends a physical velocity exactly as the padded-grid
    generators clamp their coordinates (numpy and torch alike)."""
    import numpy as np
    from paper_1502_07266_gb300 import helm, workloads as W
    n, b = 7, 3
    full = W.velocity_lens(n, b)
    phys = full[b:b + n, b:b + n, b:b + n]
    assert np.array_equal(helm.pad_velocity(phys, b), full)
    torch = pytest.importorskip("torch")
    t = helm.pad_velocity(torch.from_numpy(phys), b)
    assert np.array_equal(t.numpy(), full)


def test_default_options_match_the_header():
    """helm_default_opts (host only) fills the documented defaults, and the
    binding's struct has the header's layout: a C program compiled against
    include/helm.h reports the size and every field offset."""
    import ctypes
    import shutil
    import subprocess
    import tempfile
    from paper_1502_07266_gb300 import helm
    o = helm.helm_default_opts()
    assert (o.precision, o.b_aux, o.restart, o.maxit, o.pml_C, o.rhs_per_cta, o.schedule) == \
        (helm.HELM_FP32, 0, 30, 300, 10.0, 0, helm.HELM_ONE_FRONT)
    assert (o.apply_form, o.debug_unmet_wait, o.wait_cycles) == (helm.HELM_CHAIN, 0, 0)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in helm.helm_opts._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"helm.h\"\nint main(void){printf(\"%zu\", sizeof(helm_opts));"
    src += "".join(f'printf(" %zu", offsetof(helm_opts, {f}));' for f in fields) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "t.c"), "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), os.path.join(d, "t.c"), "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(helm.helm_opts)] + [getattr(helm.helm_opts, f).offset for f in fields]
    assert got == want


def test_tune_structs_match_the_header():
    """helm_candidate / helm_tune_result: the binding's layout is the C layout."""
    import shutil
    import subprocess
    import tempfile
    from paper_1502_07266_gb300 import helm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = [("helm_candidate", helm.helm_candidate), ("helm_tune_result", helm.helm_tune_result)]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"helm.h\"\nint main(void){"
    want = []
    for cname, cls in checks:
        src += f'printf(" %zu", sizeof({cname}));'
        want.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            src += f'printf(" %zu", offsetof({cname}, {f}));'
            want.append(getattr(cls, f).offset)
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "t.c"), "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), os.path.join(d, "t.c"), "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want


def test_tune_rejects_bad_arguments(libpath):
    """helm_tune validates its arguments before any device work."""
    from paper_1502_07266_gb300 import helm
    L = helm.lib()
    cands = (helm.helm_candidate * 1)(helm.helm_candidate(1, helm.HELM_CHAIN, helm.HELM_FP32, 0, 0))
    best = ctypes.c_int(0)
    assert L.helm_tune(None, 1.0, 7, 3, None, cands, 1, ctypes.c_void_p(16), 1, 1e-6, 0.0, None,
                       ctypes.byref(best), None) == helm.HELM_EINVAL
    assert L.helm_tune(ctypes.c_void_p(16), 1.0, 7, 3, None, cands, 0, ctypes.c_void_p(16), 1, 1e-6, 0.0, None,
                       ctypes.byref(best), None) == helm.HELM_EINVAL
    assert L.helm_tune(ctypes.c_void_p(16), 1.0, 7, 3, None, cands, 1, ctypes.c_void_p(16), 1, -1.0, 0.0, None,
                       ctypes.byref(best), None) == helm.HELM_EINVAL


def test_tune_binding_marshals_schedule_candidates(libpath):
    """The binding turns (d, form, precision[, schedule, b_aux]) tuples into the C
    candidate struct; a null velocity is rejected before any device work."""
    from paper_1502_07266_gb300 import helm
    with pytest.raises(helm.HelmError) as e:
        helm.helm_tune(0, 1.0, 7, 3, 16, 1, [(1, "dense", "split_fp16", "two_front", 2), (2, "chain", "fp32")])
    assert e.value.code == helm.HELM_EINVAL
    c = helm.helm_candidate(1, helm.HELM_DENSE, helm.HELM_SPLIT_FP16, helm.HELM_TWO_FRONT, 2)
    assert (c.d, c.apply_form, c.precision, c.schedule, c.b_aux) == (1, helm.HELM_DENSE, helm.HELM_SPLIT_FP16,
                                                                     helm.HELM_TWO_FRONT, 2)
