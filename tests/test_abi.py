"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/disc.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import subprocess

import numpy as np

from paper_1204_6295_b300 import disc


def test_library_exports_every_header_function():
    names = disc.header_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", disc.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(disc._lib, n)


def test_library_targets_sm_103a():
    from paper_1204_6295_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _header_struct_fields(name):
    """(type, field, count) of a C struct typedef in include/disc.h, comments removed."""
    import re
    text = open(disc.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{(.*?)\}\s*" + name + ";", text, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.fullmatch(r"(\w+) (.+)", decl)
        ctype = m.group(1)
        for item in m.group(2).split(","):
            item = item.strip()
            a = re.fullmatch(r"(\w+)(?:\[(\w+)\])?", item)
            count = a.group(2)
            if count is not None and not count.isdigit():
                count = str(getattr(disc, count.replace("DISC_", ""), None) or disc.MAX_LEVELS)
            out.append((ctype, a.group(1), int(count) if count else 1))
    return out


def test_params_struct_matches_header():
    """The binding's disc_params mirrors the header field by field (names, types,
    array lengths), so the struct the library reads is the one Python fills."""
    ctypes_of = {"int32_t": ctypes.c_int32, "float": ctypes.c_float}
    fields = _header_struct_fields("disc_params")
    assert [f[1] for f in fields] == [f[0] for f in disc.Params._fields_]
    for (ctype, name, count), (pname, ptype) in zip(fields, disc.Params._fields_):
        base = ctypes_of[ctype]
        expect = base * count if count > 1 else base
        assert ctypes.sizeof(ptype) == ctypes.sizeof(expect), name
        elem = ptype._type_ if issubclass(ptype, ctypes.Array) else ptype
        assert elem == base and (issubclass(ptype, ctypes.Array) == (count > 1)), name


def test_params_default_and_status_strings():
    p = disc.make_params()
    assert tuple(p.patch) == (3, 3, 3) and p.levels == 2 and p.iters[0] == 50
    assert p.stop_window == 10 and p.force_mode == disc.FORCE_THIRION
    for code in range(7):
        assert disc._lib.disc_status_str(code).decode().startswith("DISC_")
    assert disc._lib.disc_params_default(None) == 1


def test_qscale_keeps_integer_sums_in_range():
    for patch in [(3, 3, 3), (7, 7, 7), (11, 11, 11), (15, 15, 15), (25, 25, 7), (31, 31, 31)]:
        n = float(np.prod(patch))
        for mx in [0.0, 1.0, 1000.0, 3071.0, 4096.0, 1e6]:
            qs = disc.qscale(mx, patch)
            assert qs > 0 and np.log2(qs) == int(np.log2(qs))
            qmax = (mx + 1.0) * qs
            assert qmax * qmax * n < 2.0 ** 62
            assert qmax * (patch[2] + 1) < 2.0 ** 31
            # and the scale is not needlessly coarse: doubling it would overflow
            q2 = 2 * qmax
            assert q2 * q2 * n >= 2.0 ** 62 or q2 * (patch[2] + 1) >= 2.0 ** 31 or qs >= 2.0 ** 40
    assert disc.qscale(float("nan"), (3, 3, 3)) == 0.0
    assert disc.qscale(-1.0, (3, 3, 3)) == 0.0


def test_kernel_calls_reject_bad_arguments_on_host():
    p = (ctypes.c_int32 * 3)(3, 3, 3)
    even = (ctypes.c_int32 * 3)(4, 3, 3)
    f = disc._lib
    assert f.disc_k_pass_a(None, None, None, None, None, None, None, 4, 4, 4, p, 1.0, 1e-6, 0, None) == 1
    fake = ctypes.c_void_p(16)
    fake2 = ctypes.c_void_p(48)
    assert f.disc_k_pass_a(fake, fake, fake, fake2, None, None, None, 4, 4, 4, even, 1.0, 1e-6, 0, None) == 1
    assert f.disc_k_pass_a(fake, fake, fake, fake2, None, None, None, 0, 4, 4, p, 1.0, 1e-6, 0, None) == 2
    assert f.disc_k_pass_a(fake, fake, fake, fake2, None, None, None, 4, 4, 4, p, 1.0, 1e-6, 7, None) == 1
    assert f.disc_k_gauss(fake, fake, 4, 4, 4, 1.0, 0, None) == 1          # u aliases r
    assert f.disc_k_gauss(fake, ctypes.c_void_p(32), 4, 4, 4, -1.0, 0, None) == 1
    assert f.disc_k_static_norm(fake, fake, 4, 4, 4, even, 1.0, 1e-6, None) == 1
    assert f.disc_k_downsample2(fake, fake, 0, 1, 1, None) == 2
    assert f.disc_create(None, 0, None, None) == 1
    bad = disc.make_params()
    bad.patch[0] = 2
    h = ctypes.c_void_p()
    assert f.disc_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    bad = disc.make_params()
    bad.gauss_sigma = 0.0
    assert f.disc_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    assert f.disc_destroy(None) == 0
    assert f.disc_iterate(None, 1, None, None) == 1
