"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/chamfer.h declares, and shares no code with the oracle."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chamfer.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ch_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2307_03043_gb300 import build
    return build.build()


def test_header_declares_the_path(built):
    names = _declared()
    for n in ("ch_crude_nn", "ch_sample", "ch_sampled_nn", "ch_estimate", "ch_exact", "ch_serve_create",
              "ch_serve_submit", "ch_serve_wait", "ch_hash_keys"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(ch_[a-z0-9_]+)\b", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binding_covers_header(built):
    from paper_2307_03043_gb300 import binding
    so = binding.lib()
    for n in _declared():
        assert hasattr(so, n)
    assert set(binding.SIGNATURES) == _declared()


def test_library_shares_no_code_with_oracle(built):
    out = subprocess.run(["nm", "-D", built], capture_output=True, text=True, check=True).stdout
    assert not re.search(r"\bor_[a-z0-9_]+\b", out)
    ldd = subprocess.run(["ldd", built], capture_output=True, text=True).stdout
    assert "oracle" not in ldd
    csrc = os.path.join(ROOT, "paper_2307_03043_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f


def test_build_targets_sm_103a_only():
    from paper_2307_03043_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-use_fast_math" not in build.NVCC_FLAGS and "-ftz=false" in build.NVCC_FLAGS


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2307_03043_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(binding.ChamferError):
        binding.lib()


def test_default_params_match_the_header(built):
    """ch_default_params fills the defaults include/chamfer.h documents (a host
    call: no device is touched)."""
    import ctypes
    from paper_2307_03043_gb300 import binding as ch
    p = ch.ch_est_params()
    ctypes.memset(ctypes.byref(p), 0xAB, ctypes.sizeof(p))
    ch.lib().ch_default_params(ctypes.byref(p))
    h = p.hash
    assert (h.metric, h.levels, h.proj_dim, h.top_exp, h.hash_seed, h.group) == \
        (ch.CH_L1, 10, 16, ch.CH_TOP_EXP_AUTO, 0, ch.CH_GROUP_HASH)
    assert h.window in (0, 1) and h.repeats in (0, 1) and h.family == 0  # Fig. 2's single structure, grids
    assert (p.eps, p.T, p.sample_seed, p.screen, p.rerank_k, p.sampling) == \
        (0.1, 0, 0, ch.CH_SCREEN_AUTO, 8, ch.CH_SAMPLING_IMPORTANCE)


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every struct the binding mirrors has the size and field offsets that a C
    compiler gives the header's declaration (gcc on this host)."""
    import ctypes
    import shutil
    from paper_2307_03043_gb300 import binding as ch
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [ch.ch_hash_params, ch.ch_est_params, ch.ch_est_report, ch.ch_serve_config, ch.ch_serve_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chamfer.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'  printf("{s.__name__} size %zu\\n", sizeof({s.__name__}));')
        for f in s._fields_:
            lines.append(f'  printf("{s.__name__} {f[0]} %zu\\n", offsetof({s.__name__}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = ln.split()
        got[(name, field)] = int(value)
    for s in structs:
        assert got[(s.__name__, "size")] == ctypes.sizeof(s), s.__name__
        for f in s._fields_:
            assert got[(s.__name__, f[0])] == getattr(s, f[0]).offset, (s.__name__, f[0])


NULL_CTX_CALLS = ["ch_ctx_sync", "ch_set_create", "ch_set_prepare", "ch_top_exp", "ch_hash_keys", "ch_crude_nn",
                  "ch_sample", "ch_sampled_nn", "ch_estimate", "ch_estimate_batch", "ch_estimate_sym", "ch_exact",
                  "ch_ctx_set_wait_cycles", "ch_set_embed"]


@pytest.mark.parametrize("name", NULL_CTX_CALLS)
def test_null_context_is_an_argument_error(built, name):
    """Every call that takes a context answers CH_EINVAL to a NULL one, before
    any device work (the header's error contract; runs without a GPU)."""
    import ctypes
    from paper_2307_03043_gb300 import binding as ch
    fn = getattr(ch.lib(), name)
    args = []
    for t in fn.argtypes:
        if t in (ctypes.c_double, ctypes.c_float):
            args.append(0.0)
        elif issubclass(t, ctypes._SimpleCData) and t is not ctypes.c_void_p and t._type_ not in "zPO":
            args.append(0)
        else:
            args.append(None)
    assert fn(*args) == ch.CH_EINVAL


def test_context_without_a_device_is_a_cuda_error(built):
    """With no CUDA device, ch_ctx_create reports CH_ECUDA, frees what it made
    and leaves *out as it was (set on success only)."""
    import ctypes
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2307_03043_gb300 import binding as ch
    out = ctypes.c_void_p(1234)
    assert ch.lib().ch_ctx_create(0, None, ctypes.byref(out)) == ch.CH_ECUDA
    assert out.value == 1234
    assert ch.lib().ch_ctx_create(0, None, None) == ch.CH_EINVAL
