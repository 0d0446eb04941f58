"""CPU checks of the C ABI: the library loads, exports every entry point that
include/hmm.h and include/hmm_dns.h declare, and rejects invalid parameters on
the host (no GPU needed: validation happens before any CUDA call)."""
import ctypes
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_09463_gb300 import build, load_library
    build()
    return load_library()


def _declared(header="hmm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmm_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2108_09463_gb300 import EXPORTED
    decl = _declared()
    assert decl == sorted(EXPORTED)
    for name in decl:
        assert hasattr(lib, name), name


def test_exports_every_declared_dns_symbol(lib):
    from paper_2108_09463_gb300 import EXPORTED_DNS
    decl = _declared("hmm_dns.h")
    assert decl == sorted(EXPORTED_DNS)
    for name in decl:
        assert hasattr(lib, name), name


def test_headers_cover_every_export():
    """Every .h under include/ is bound: no header declares an unbound symbol."""
    from paper_2108_09463_gb300 import EXPORTED, EXPORTED_DNS
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        names |= set(_declared(f))
    assert names == set(EXPORTED) | set(EXPORTED_DNS)


def _struct_fields(src, name):
    body = re.search(r"typedef struct \{([^{}]*)\} " + name + ";", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.replace("const", " ").replace("*", " ").strip()
        if not decl:
            continue
        # drop the type (first token), keep the declarators
        decl = decl.split(None, 1)[1]
        out += [re.sub(r"\[\d+\]", "", v).strip() for v in decl.split(",")]
    return out


def test_struct_layout_matches_header():
    """The ctypes mirror has the field order of hmm_params / hmm_coef_term."""
    from paper_2108_09463_gb300._lib import HmmCoefTerm, HmmParams
    src = open(os.path.join(ROOT, "include", "hmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    assert [f[0] for f in HmmParams._fields_] == _struct_fields(src, "hmm_params")
    assert [f[0] for f in HmmCoefTerm._fields_] == _struct_fields(src, "hmm_coef_term")


def test_dns_struct_layout_matches_header():
    from paper_2108_09463_gb300._lib import HmmDnsParams
    src = open(os.path.join(ROOT, "include", "hmm_dns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    assert [f[0] for f in HmmDnsParams._fields_] == _struct_fields(src, "hmm_dns_params")


def _init(lib, cfg, **over):
    from paper_2108_09463_gb300._lib import make_params
    p, keep = make_params(cfg)
    for k, v in over.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    st = lib.hmm_init(ctypes.byref(p), None, ctypes.byref(h))
    msg = lib.hmm_last_error(None).decode()
    if st == 0:
        lib.hmm_destroy(h)
    return st, msg


@pytest.mark.parametrize("over,needle", [
    (dict(dim=4), "dim"), (dict(alpha=0.0), "alpha"), (dict(alpha=1.5), "alpha"),
    (dict(alpha_micro=-1.0), "alpha_micro"), (dict(stencil_order=3), "stencil_order"),
    (dict(interp_order=6), "interp_order"), (dict(precision=5), "precision"),
    (dict(micro_steps=0), "micro_steps"), (dict(box_n=5), "box_n"), (dict(box_n=300), "box_n"),
    (dict(eps=-1.0), "eps"), (dict(pts_per_eps=0.0), "pts_per_eps"), (dict(n_terms=9), "n_terms"),
    (dict(model=2), "model"),
])
def test_invalid_params_rejected_on_host(lib, over, needle):
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=24, micro_steps=10)
    st, msg = _init(lib, cfg, **over)
    assert st == 1, (st, msg)
    assert needle in msg


def test_single_micro_step_rejected_on_host(lib):
    """M = 1: both time nodes are end points of K0's support, so every weight vanishes."""
    st, msg = _init(lib, W.config("c2_2d", n_macro=(6, 6, 1), box_n=24, micro_steps=1))
    assert st == 1 and "time weights" in msg, (st, msg)


def test_averaging_box_must_avoid_ring(lib):
    cfg = W.config("c2_2d", n_macro=(8, 8, 1), box_n=20, micro_steps=10)  # mu = 0.8 mu' reaches the ring
    st, msg = _init(lib, cfg)
    assert st == 1 and "ring" in msg


def test_null_arguments(lib):
    assert lib.hmm_init(None, None, None) == 1
    assert lib.hmm_micro_batch(None, None, None) == 7
    assert lib.hmm_macro_step(None, None, 1) == 7
    assert lib.hmm_macro_step_wave(None, None, 0, 1) == 7
    assert lib.hmm_fp32_fma_rate(1, None) == 1          # checked before any CUDA call
    assert lib.hmm_fp32_fma_rate(2, ctypes.byref(ctypes.c_double())) == 1
    lib.hmm_destroy(None)


def _dns_init(lib, cfg, **over):
    from paper_2108_09463_gb300._lib import make_dns_params
    p, keep = make_dns_params(cfg)
    for k, v in over.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    st = lib.hmm_dns_init(ctypes.byref(p), None, ctypes.byref(h))
    msg = lib.hmm_dns_last_error(None).decode()
    if st == 0:
        lib.hmm_dns_destroy(h)
    return st, msg


@pytest.mark.parametrize("over,needle", [
    (dict(dim=3), "dim"), (dict(alpha=-0.1), "alpha"), (dict(alpha=1.5), "alpha"),
    (dict(stencil_order=3), "stencil_order"), (dict(precision=2), "precision"),
    (dict(eps=0.0), "eps"), (dict(n_terms=9), "n_terms"), (dict(L=0.0), "L"),
    (dict(c0=0.2), "a^eps <= 0"),
])
def test_dns_invalid_params_rejected_on_host(lib, over, needle):
    cfg = W.dns_config("dns_quasi2d", n=(40, 36, 1))
    st, msg = _dns_init(lib, cfg, **over)
    assert st == 1, (st, msg)
    assert needle in msg


def test_dns_grid_limits(lib):
    cfg = W.dns_config("dns_quasi2d", n=(3, 36, 1))
    st, msg = _dns_init(lib, cfg)
    assert st == 1 and "n[k]" in msg
    cfg = W.dns_config("dns_quasi2d", n=(1 << 16, 1 << 16, 1))
    st, msg = _dns_init(lib, cfg)
    assert st == 1 and "too many" in msg


def test_dns_null_arguments(lib):
    assert lib.hmm_dns_init(None, None, None) == 1
    assert lib.hmm_dns_step(None, None, 1) == 7
    assert lib.hmm_dns_reset(None) == 7
    lib.hmm_dns_destroy(None)


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++17")])
def test_headers_compile_on_their_own(tmp_path, lang, std):
    """The public headers are plain C (no CUDA or torch types) and compile as C99 and C++17."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "use_headers.c"
    src.write_text('#include "hmm.h"\n#include "hmm_dns.h"\nint main(void) { return (int)HMM_OK; }\n')
    r = subprocess.run([cc, "-x", lang, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_gets_a_host_side_refusal(tmp_path, lib):
    """A C program (no Python) links libhmm_gb300.so, fills hmm_params with an invalid
    dimension and gets HMM_ERR_INVALID_ARG with a message from hmm_last_error(NULL):
    parameter validation runs on the host, before any CUDA call."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    from paper_2108_09463_gb300 import build
    libdir = os.path.dirname(build())
    src = tmp_path / "refusal.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "hmm.h"
int main(void) {
  hmm_params p;
  void* h = NULL;
  memset(&p, 0, sizeof p);
  p.dim = 7;
  hmm_status s = hmm_init(&p, NULL, &h);
  printf("%d|%s\n", (int)s, hmm_last_error(NULL));
  return s == HMM_ERR_INVALID_ARG && h == NULL ? 0 : 1;
}
''')
    exe = tmp_path / "refusal"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lhmm_gb300", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    status, msg = r.stdout.strip().split("|", 1)
    assert int(status) == 1 and "dim" in msg
