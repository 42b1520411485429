"""The C-ABI library builds, loads and exports every symbol include/lb.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lb\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_0911_0459_gb300 import build
    return build.build()


def test_header_declares_the_interface():
    names = declared_functions()
    for n in ("lb_create", "lb_step", "lb_fields", "lb_filled_length", "lb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches_header(libpath):
    from paper_0911_0459_gb300 import lb
    lib = lb.library()
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(lb.exported_symbols()) <= set(declared_functions())


def test_struct_layouts_match_header(libpath, tmp_path):
    """Compile a C probe of sizeof/offsetof and compare with the ctypes structs."""
    from paper_0911_0459_gb300 import lb
    probe = tmp_path / "p.c"
    fields = {"lb_walls": [f[0] for f in lb.LbWalls._fields_], "lb_params": [f[0] for f in lb.LbParams._fields_],
              "lb_grid": [f[0] for f in lb.LbGrid._fields_], "lb_alloc": [f[0] for f in lb.LbAlloc._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lb.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "p"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    py = {"lb_walls": lb.LbWalls, "lb_params": lb.LbParams, "lb_grid": lb.LbGrid, "lb_alloc": lb.LbAlloc}
    for s, cls in py.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fields[s]:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_workload_wall_gradient_matches_oracle_closed_form():
    """The input conversion theta -> d_n phi|_b of the workloads (bisection) and the oracle's
    own root of the same closed form agree to rounding."""
    import workloads as W
    from oracle import analysis as an
    for th in (30.0, 45.0, 60.0, 80.0):
        for A in (0.03, 0.04, 0.05):
            assert abs(W.binary_wall_gradient(th, A, A) - an.binary_wall_gradient_for_angle(th, A, A)) < 1e-14


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_0911_0459_gb300 import lb
    monkeypatch.setattr(lb, "_lib", None)
    monkeypatch.setattr(lb, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lb.library()


def _create_status(lib, grid, walls, params):
    ctx = ctypes.c_void_p()
    st = lib.lb_create(ctypes.byref(grid), ctypes.byref(walls), ctypes.byref(params), None, None, ctypes.byref(ctx))
    return st, ctx.value, lib.lb_last_error(None).decode()


def test_create_rejects_invalid_arguments_before_any_cuda_call(libpath):
    """Argument checks of lb_create run on the host before the first CUDA call: every
    invalid lattice returns LB_ERR_ARG with a message and no context (no GPU needed)."""
    import workloads as W
    from paper_0911_0459_gb300 import lb
    lib = lb.library()
    cap = W.Capillary("v", 96, 24, 24, 64, 3, 18, 8, 6, W.binary_params(), theta_deg=45.0)

    def edits():
        yield "nx < 3", lambda g, w, p: setattr(g, "nx", 2)
        yield "more than 2^31 - 1 nodes", lambda g, w, p: (setattr(g, "nx", 65536), setattr(g, "ny", 32769))
        yield "moments above 715827882 nodes", lambda g, w, p: (setattr(g, "nx", 65536), setattr(g, "ny", 10923),
                                                               setattr(p, "storage", lb.STORAGE_MOMENTS))
        yield "liquid-gas in FP16", lambda g, w, p: (setattr(p, "model", 0), setattr(p, "storage", lb.STORAGE_F16DEV))
        yield "liquid-gas in FP16 moments", lambda g, w, p: (setattr(p, "model", 0),
                                                             setattr(p, "storage", lb.STORAGE_MOMENTS_F16))
        yield "liquid-gas with g eliminated", lambda g, w, p: (setattr(p, "model", 0),
                                                               setattr(p, "storage", lb.STORAGE_F32_GELIM))
        yield "g eliminated above 429496729 nodes", lambda g, w, p: (setattr(g, "nx", 65536), setattr(g, "ny", 6554),
                                                                     setattr(p, "storage", lb.STORAGE_F32_GELIM))
        yield "liquid-gas in blocks", lambda g, w, p: (setattr(p, "model", 0),
                                                       setattr(p, "storage", lb.STORAGE_F32_BLOCKED))
        yield "block storage above 238609280 nodes", lambda g, w, p: (setattr(g, "nx", 65536), setattr(g, "ny", 3641),
                                                                      setattr(p, "storage", lb.STORAGE_F32_BLOCKED))
        yield "liquid-gas in FP16 blocks", lambda g, w, p: (setattr(p, "model", 0),
                                                            setattr(p, "storage", lb.STORAGE_F16_BLOCKED))
        yield "FP16 blocks above 226050880 nodes", lambda g, w, p: (setattr(g, "nx", 65536), setattr(g, "ny", 3450),
                                                                    setattr(p, "storage", lb.STORAGE_F16_BLOCKED))
        yield "unknown storage", lambda g, w, p: setattr(p, "storage", 9)
        yield "tube longer than the grid", lambda g, w, p: setattr(w, "tube_len", 97)
        yield "band as tall as the grid", lambda g, w, p: setattr(w, "tube_h", 24)
        yield "band of one row", lambda g, w, p: setattr(w, "tube_h", 1)
        yield "one reservoir column", lambda g, w, p: setattr(w, "tube_len", 95)
        yield "wall gradient NaN", lambda g, w, p: setattr(w, "wall_grad", float("nan"))
        yield "viscosity table of one entry", lambda g, w, p: setattr(p, "nu_table", 1)
        yield "zero liquid viscosity", lambda g, w, p: setattr(p, "nu_l", 0.0)
        yield "negative mobility", lambda g, w, p: setattr(p, "M", -0.1)

    for what, edit in edits():
        g, w, p = lb._structs_for(cap)
        edit(g, w, p)
        st, ctx, msg = _create_status(lib, g, w, p)
        assert st == lb.LB_ERR_ARG and ctx is None and msg, what
    # a mobility of zero is valid: the check is on the sign
    g, w, p = lb._structs_for(cap)
    p.M = 0.0
    p.nu_table = -1
    assert _create_status(lib, g, w, p)[0] == lb.LB_ERR_ARG


def test_batch_create_rejects_invalid_arguments_before_any_cuda_call(libpath):
    import workloads as W
    from paper_0911_0459_gb300 import lb
    lib = lb.library()
    caps = [W.Capillary("b", 96, 24, 24, 64, 3, 18, 8, 6, W.binary_params(), theta_deg=45.0),
            W.Capillary("c", 104, 30, 24, 72, 3, 22, 8, 6, W.binary_params(), theta_deg=60.0)]

    def status(edit=None, n=None):
        s = [lb._structs_for(c) for c in caps]
        if edit:
            edit(s)
        m = len(s) if n is None else n
        G = (lb.LbGrid * len(s))(*[x[0] for x in s])
        Wl = (lb.LbWalls * len(s))(*[x[1] for x in s])
        P = (lb.LbParams * len(s))(*[x[2] for x in s])
        out = ctypes.c_void_p()
        st = lib.lb_batch_create(m, G, Wl, P, None, None, ctypes.byref(out))
        return st, out.value, lib.lb_batch_last_error(None).decode()

    def setp(i, k, v):
        return lambda s: setattr(s[i][2], k, v)

    cases = {
        "no lattices": (None, 0),
        "unknown storage": (lambda s: [setattr(x[2], "storage", 9) for x in s], None),
        "liquid-gas lattice": (setp(1, "model", 0), None),
        "mixed storages": (setp(1, "storage", lb.STORAGE_F64), None),
        "moments above 715827882 nodes": (lambda s: ([setattr(x[2], "storage", lb.STORAGE_MOMENTS) for x in s],
                                                    setattr(s[1][0], "nx", 65536), setattr(s[1][0], "ny", 10923),
                                                    setattr(s[1][1], "tube_len", 0)), None),
        "wall gradient NaN": (lambda s: setattr(s[0][1], "wall_grad", float("nan")), None),
        "FP16 moments in a batch": (lambda s: [setattr(x[2], "storage", lb.STORAGE_MOMENTS_F16) for x in s], None),
        "g eliminated in a batch": (lambda s: [setattr(x[2], "storage", lb.STORAGE_F32_GELIM) for x in s], None),
        "block storage above 238609280 nodes": (lambda s: ([setattr(x[2], "storage", lb.STORAGE_F32_BLOCKED) for x in s],
                                                          setattr(s[1][0], "nx", 65536), setattr(s[1][0], "ny", 3641),
                                                          setattr(s[1][1], "tube_len", 0)), None),
        "FP16 blocks above 226050880 nodes": (lambda s: ([setattr(x[2], "storage", lb.STORAGE_F16_BLOCKED) for x in s],
                                                        setattr(s[1][0], "nx", 65536), setattr(s[1][0], "ny", 3450),
                                                        setattr(s[1][1], "tube_len", 0)), None),
        "negative mobility": (setp(0, "M", -1.0), None),
        "viscosity table of one entry": (setp(1, "nu_table", 1), None),
        "tube longer than the grid": (lambda s: setattr(s[1][1], "tube_len", 200), None),
    }
    for what, (edit, n) in cases.items():
        st, h, msg = status(edit, n)
        assert st == lb.LB_ERR_ARG and h is None and msg, what


def test_fp64_rate_rejects_a_null_output_before_any_cuda_call(libpath):
    from paper_0911_0459_gb300 import lb
    assert lb.library().lb_fp64_fma_rate(None, None) == lb.LB_ERR_ARG


def test_mlp_create_rejects_invalid_shapes_before_any_cuda_call(libpath):
    """lb_mlp_create checks the network shape on the host: the largest batch is 65535 row
    tiles of 64 (the GEMMs put row tiles on the grid's y dimension)."""
    from paper_0911_0459_gb300 import lb
    from paper_0911_0459_gb300.mlp import _lib
    L = _lib()
    bad = [(4, 256, 64, 5, 65535 * 64 + 1), (4, 256, 64, 5, 0), (17, 256, 64, 5, 4096), (4, 100, 64, 5, 4096),
           (4, 256, 60, 5, 4096), (4, 256, 64, 17, 4096), (4, 2048, 64, 5, 4096), (0, 256, 64, 5, 4096)]
    for shape in bad:
        out = ctypes.c_void_p()
        st = L.lb_mlp_create(*shape, 0, None, None, ctypes.byref(out))
        assert st == lb.LB_ERR_ARG and out.value is None, shape
        assert L.lb_mlp_last_error(None).decode()


def test_noalloc_rejects_invalid_arguments_before_any_cuda_call(libpath):
    """lb_filled_length_noalloc checks its arguments on the host and returns LB_ERR_ARG
    before its first CUDA call (so this runs without a GPU; the device pointers below are
    never dereferenced): NULL pointers, block counts outside [1, LB_NOALLOC_MAX_BLOCKS],
    the moment storage (it keeps no populations), a liquid-gas lattice in FP16 or in 32-node blocks, block lattices above their node limits, a binary
    call without g, an FP16 call without g0, and liquid-gas densities that are not finite
    with rho_l > rho_g (its liquid fraction divides by rho_l - rho_g)."""
    import workloads as W
    from paper_0911_0459_gb300 import lb
    lib = lb.library()
    fn = lib.lb_filled_length_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lb.LbGrid), ctypes.POINTER(lb.LbWalls), ctypes.POINTER(lb.LbParams),
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    fake = ctypes.c_void_p(0x1000)
    binary = W.Capillary("v", 96, 24, 24, 64, 3, 18, 8, 6, W.binary_params(), theta_deg=45.0)
    lg = W.config_lg_256x32()

    def call(cap, f=fake, g=fake, g0=fake, nblocks=64, out=fake, **edit):
        gr, w, p = lb._structs_for(cap)
        for k, v in edit.items():
            setattr(p, k, v)
        return fn(ctypes.byref(gr), ctypes.byref(w), ctypes.byref(p), f, g, g0, nblocks, out, None)

    cases = {
        "f NULL": call(binary, f=None),
        "out NULL": call(binary, out=None),
        "no blocks": call(binary, nblocks=0),
        "too many blocks": call(binary, nblocks=2049),
        "moment storage": call(binary, storage=lb.STORAGE_MOMENTS),
        "liquid-gas in blocks": call(lg, storage=lb.STORAGE_F32_BLOCKED),
        "liquid-gas in FP16 blocks": call(lg, storage=lb.STORAGE_F16_BLOCKED),
        "unknown storage": call(binary, storage=8),
        "liquid-gas in FP16": call(lg, storage=lb.STORAGE_F16DEV),
        "binary without g": call(binary, g=None),
        "FP16 without g0": call(binary, g0=None, storage=lb.STORAGE_F16DEV),
        "rho_l == rho_g": call(lg, rho_l=3.0, rho_g=3.0),
        "rho_l < rho_g": call(lg, rho_l=2.59, rho_g=4.54),
        "rho_l NaN": call(lg, rho_l=float("nan")),
        "rho_g infinite": call(lg, rho_g=float("-inf")),
        "unknown model": call(binary, model=5),
        "FP32 blocks above 238609280 nodes": call(W.periodic_box(65536, 3641, W.binary_params()), g=None,
                                                  storage=lb.STORAGE_F32_BLOCKED),
        "FP16 blocks above 226050880 nodes": call(W.periodic_box(65536, 3450, W.binary_params()), g=None,
                                                  storage=lb.STORAGE_F16_BLOCKED),
    }
    bad = {k: v for k, v in cases.items() if v != lb.LB_ERR_ARG}
    assert not bad, bad
