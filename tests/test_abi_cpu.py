"""C-ABI checks that need no GPU: the library loads, exports every symbol the header
declares, and rejects invalid plan descriptions before touching the device."""
import os
import re

import numpy as np
import pytest

import synth
from paper_2306_08514_gb300._abi import METHODS as M_

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "libsrp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def S():
    import paper_2306_08514_gb300 as S
    if not os.path.exists(S.LIB_PATH):
        from paper_2306_08514_gb300 import build
        build.build()
    S.lib()
    return S


def test_library_exports_every_declared_symbol(S):
    syms = _header_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(S.lib(), name), name
    assert set(syms) == set(S.SIGNATURES)


@pytest.mark.parametrize("bad", [
    dict(M=1), dict(N=500), dict(N=128), dict(N=4096), dict(fs=0.0), dict(c=-1.0),
    dict(window=7), dict(n_aux=-1), dict(max_frames=0), dict(method=9),
    dict(method=1, rank=0), dict(method=1, rank=65), dict(method=2, taps=0.0),
    dict(method=2, taps=1e9), dict(precision=7), dict(precision=-1), dict(far_field=2), dict(far_field=1),
    dict(method=4, n_aux=0), dict(method=5, rank=0), dict(method=5, rank=65), dict(method=6),
])
def test_invalid_desc_is_rejected_on_the_host(S, bad):
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (5, 5))
    kw = dict(mic_xyz=mics, grid_xyz=grid, fs=16000.0, N=512)
    kw.update({k: v for k, v in bad.items() if k in ("fs", "N")})
    d = S.make_desc(kw["mic_xyz"], kw["grid_xyz"], kw["fs"], kw["N"],
                    method=bad.get("method", 0), rank=bad.get("rank", 4), taps=bad.get("taps", 1.0),
                    precision=bad.get("precision", 0), c=bad.get("c", 340.0),
                    n_aux=bad.get("n_aux", 2), max_frames=bad.get("max_frames", 8))
    if "M" in bad:
        d.M = bad["M"]
    if "window" in bad:
        d.window = bad["window"]
    if "far_field" in bad:  # 2 is out of range; 1 with a grid of locations, not unit vectors
        d.far_field = bad["far_field"]
    with pytest.raises(S.SrpError) as e:
        S.srp_plan_create(d, None)
    assert e.value.status in (S.SRP_EINVAL, S.SRP_EUNSUPPORTED)
    assert S.srp_last_error()


@pytest.mark.parametrize("J,precision", [(65535 * 1024 + 1, "bf16"), (65535 * 128 + 1, "fp32")])
def test_grid_larger_than_the_launch_grids_is_rejected(S, J, precision):
    """J beyond what the map kernels' grids cover (65535 block rows of 1024 cells, or 128 for
    the FP32 FFMA GEMM) is refused before grid_xyz is read, so a small array serves here."""
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (5, 5))
    d = S.make_desc(mics, grid, 16000.0, 512, precision=precision)
    d.J = J
    for call in (lambda: S.srp_plan_create(d, None), lambda: S.srp_plan_estimate_bytes(d)):
        with pytest.raises(S.SrpError) as e:
            call()
        assert e.value.status == S.SRP_EINVAL and "J" in str(e.value)


def test_window_wider_than_frame_is_rejected(S):
    mics = synth.mics_square() * 40.0
    grid = synth.grid_plane((0, 0), (4, 4), (5, 5))
    d = S.make_desc(mics, grid, 16000.0, 256)
    with pytest.raises(S.SrpError) as e:
        S.srp_plan_create(d, None)
    assert e.value.status == S.SRP_EINVAL
    assert "N_p" in S.srp_last_error()


def test_null_arguments(S):
    assert S.lib().srp_map(None, None, 1, None, None, None) == S.SRP_EINVAL
    assert S.lib().srp_plan_info(None, None) == S.SRP_EINVAL
    S.srp_destroy(None)


def test_plan_estimate_needs_no_gpu(S):
    """srp_plan_estimate_bytes (admission by footprint) is host arithmetic: it scales with the
    operands a plan would hold."""
    mics = synth.mics_uca(8, 0.05, (2.5, 2.0, 1.5))
    grid = synth.grid_box((0, 0, 0), (5.0, 4.0, 3.0), 0.1)
    conv16 = S.srp_plan_estimate_bytes(S.make_desc(mics, grid, 16000.0, 512, precision="bf16", max_frames=64))
    conv32 = S.srp_plan_estimate_bytes(S.make_desc(mics, grid, 16000.0, 512, max_frames=64))
    slri = S.srp_plan_estimate_bytes(S.make_desc(mics, grid, 16000.0, 512, method="slri", rank=16,
                                                 max_frames=64))
    J, P, N = grid.shape[0], 28, 512
    assert abs(conv32 - 2 * conv16) < 0.02 * conv32
    assert J * P * N * 4 <= conv32 <= 1.1 * J * P * N * 4
    assert slri < conv16 / 50
    # TF32 operands are 4 bytes, the x3 precisions hold hi and lo planes
    est = {p: S.srp_plan_estimate_bytes(S.make_desc(mics, grid, 16000.0, 512, precision=p, max_frames=64))
           for p in ("tf32", "bf16x3", "fp16x3", "tf32x3")}
    assert abs(est["tf32"] - conv32) < 0.02 * conv32
    assert abs(est["bf16x3"] - 2 * conv16) < 0.02 * conv32 and est["bf16x3"] == est["fp16x3"]
    assert abs(est["tf32x3"] - 2 * conv32) < 0.02 * conv32


def test_allocation_failure_hook_checks_its_arguments(S):
    """srp_debug_fail_allocations is host bookkeeping (no GPU): negative counts are refused,
    and n = 0 clears the injection."""
    for after, n in ((-1, 1), (0, -1)):
        with pytest.raises(S.SrpError) as e:
            S.srp_debug_fail_allocations(after, n)
        assert e.value.status == S.SRP_EINVAL
    S.srp_debug_fail_allocations(3, 2)
    S.srp_debug_fail_allocations(0, 0)


def _fnv1a64(b):
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_plan_file_is_checked_before_any_gpu_work(S, tmp_path):
    """srp_plan_create_from_file refuses a missing file, a foreign file, a damaged file and a
    well-formed file made for other inputs, on the host (no GPU is touched)."""
    import struct
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (10, 10))
    desc = S.make_desc(mics, grid, 16000.0, 512, method="slri", rank=4)

    def refused(path, what):
        with pytest.raises(S.SrpError) as e:
            S.srp_plan_create_from_file(desc, path)
        assert e.value.status == S.SRP_EINVAL and what in str(e.value), str(e.value)

    refused(tmp_path / "missing.plan", "cannot open")
    foreign = tmp_path / "foreign.plan"
    foreign.write_bytes(b"not a plan file at all")
    refused(foreign, "not a libsrp plan file")
    body = b"SRPPLAN\0" + struct.pack("<Iiq", 1, 1, 12345) + struct.pack("<iiii", 100, 6, 0, 4)
    good_sum = body + struct.pack("<Q", _fnv1a64(body))
    other = tmp_path / "other.plan"
    other.write_bytes(good_sum)
    refused(other, "other inputs")
    damaged = tmp_path / "damaged.plan"
    damaged.write_bytes(good_sum[:-1] + bytes([good_sum[-1] ^ 1]))
    refused(damaged, "checksum")


def _fit_inputs_hash(S, desc, mics, grid):
    """The hash srp_plan_save stores: FNV-1a 64 over the fields the fit depends on, in the
    order and widths of srp_plan_desc (int32 / float64, little-endian)."""
    import struct
    sspi = desc.method == M_["sspi"]
    lowrank = desc.method in (M_["slri"], M_["lr"])
    b = struct.pack("<i", desc.M) + np.ascontiguousarray(mics, "<f8").tobytes()
    b += struct.pack("<i", desc.J) + np.ascontiguousarray(grid, "<f8").tobytes()
    b += struct.pack("<did", desc.fs, desc.N, desc.c)
    b += struct.pack("<iii", desc.n_aux, desc.method, desc.rank if lowrank else 0)
    b += struct.pack("<di", desc.taps_per_loc_pair if sspi else 0.0, desc.far_field)
    return _fnv1a64(b)


def test_plan_file_with_bad_sspi_taps_is_refused_before_any_gpu_work(S, tmp_path):
    """An SSPI plan file whose header, input hash and checksum are all right but whose taps
    would index outside the device buffers (a column outside [0, L), row pointers out of
    order, a row range that does not cover the taps) is refused on the host."""
    import struct
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (10, 10))
    desc = S.make_desc(mics, grid, 16000.0, 512, method="sspi", taps=1.0)
    J, M = grid.shape[0], mics.shape[0]
    pairs = [(m, mp) for mp in range(M - 1) for m in range(mp + 1, M)]
    Np = [int(np.floor(np.sqrt(((mics[m] - mics[mp]) ** 2).sum()) / desc.c * desc.fs)) + desc.n_aux
          for m, mp in pairs]
    P, L = len(pairs), sum(2 * n + 1 for n in Np)
    h = _fit_inputs_hash(S, desc, mics, grid)

    def plan_file(name, row_ptr, col, nnz=None, tail=b""):
        row_ptr = np.asarray(row_ptr, "<i8")
        col = np.asarray(col, "<i4")
        nnz = len(col) if nnz is None else nnz
        body = b"SRPPLAN\0" + struct.pack("<IiQ", 1, M_["sspi"], h)
        body += struct.pack("<iiii", J, P, L, 0) + struct.pack("<qq", nnz, 0)
        for a in (row_ptr, col, np.ones(len(col), "<f4")):
            body += struct.pack("<Q", a.size) + a.tobytes()
        body += tail
        path = tmp_path / name
        path.write_bytes(body + struct.pack("<Q", _fnv1a64(body)))
        return path

    rows = np.arange(J + 1)  # one tap per location
    cols = np.arange(J) % L
    # control: the unflawed file passes every file check (without a GPU the plan then fails
    # at its first CUDA call; with one it is created)
    try:
        S.srp_destroy(S.srp_plan_create_from_file(desc, plan_file("ok.plan", rows, cols)))
    except S.SrpError as e:
        assert e.status != S.SRP_EINVAL and "plan file" not in str(e), str(e)
    for name, args in [
        ("col_high", (rows, np.where(np.arange(J) == 7, L, cols))),
        ("col_negative", (rows, np.where(np.arange(J) == 0, -1, cols))),
        ("rows_unordered", (np.where(np.arange(J + 1) == 5, 9, rows), cols)),
        ("rows_start", (rows + 1, cols)),
        ("rows_short", (np.minimum(rows, J - 1), cols)),
        ("trailing", (rows, cols, None, b"\0\0\0\0")),
    ]:
        with pytest.raises(S.SrpError) as e:
            S.srp_plan_create_from_file(desc, plan_file(name + ".plan", *args))
        assert e.value.status == S.SRP_EINVAL
        assert "contents do not match its header" in str(e.value), (name, str(e.value))


def test_header_serves_a_plain_c_program(S, tmp_path):
    """include/libsrp.h compiles as strict C99 and C11 (no C++ in the interface), and a C
    program linked against libsrp.so alone sizes a plan and gets the documented host-side
    argument checks (tests/abi_consumer.c; no call needs a GPU)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = os.path.join(ROOT, "tests", "abi_consumer.c")
    lib_dir = os.path.dirname(S.LIB_PATH)
    for std in ("c99", "c11"):
        exe = str(tmp_path / f"consumer_{std}")
        subprocess.run([gcc, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe, S.LIB_PATH,
                        f"-Wl,-rpath,{lib_dir}"], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


def test_binding_structs_match_the_header_layout(S, tmp_path):
    """The ctypes structures of the Python binding have the size and field offsets that a C
    compiler gives the header's structures (a drift between include/libsrp.h and the binding
    would pass garbage across the ABI)."""
    import ctypes
    import shutil
    import subprocess
    from paper_2306_08514_gb300 import _abi as A
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"srp_plan_desc": A.srp_plan_desc, "srp_plan_info_t": A.srp_plan_info_t,
               "srp_server_desc": A.srp_server_desc, "srp_server_stats_t": A.srp_server_stats_t,
               "srp_tune_report_t": A.srp_tune_report_t}
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include \"libsrp.h\"", "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:-1]): int(l.split()[-1]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def _header_declarations():
    """(name, return type, [parameter declarations]) of every function the header declares."""
    text = open(os.path.join(ROOT, "include", "libsrp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"#.*", "", text)
    out = []
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(srp_[a-z_]+)\s*\(([^;{]*?)\)\s*;", text):
        ret = " ".join(m.group(1).split()[-3:])
        params = [p.strip() for p in m.group(3).split(",")]
        if params == ["void"]:
            params = []
        out.append((m.group(2), ret, params))
    return out


def test_binding_signatures_match_the_header(S):
    """Every entry point's ctypes signature has the header's parameter count, pointers where
    the header has pointers (or handle typedefs), and scalars of the header's width."""
    import ctypes
    decls = _header_declarations()
    assert {d[0] for d in decls} == set(S.SIGNATURES)
    scalars = {"int": ctypes.c_int, "double": ctypes.c_double, "size_t": ctypes.c_size_t,
               "float": ctypes.c_float, "long long": ctypes.c_longlong}
    handles = ("srp_plan_t", "srp_server_t")
    for name, ret, params in decls:
        restype, argtypes = S.SIGNATURES[name]
        assert len(argtypes) == len(params), name
        for p, t in zip(params, argtypes):
            ptype = re.sub(r"\b(const|restrict)\b", "", p).strip()
            if "*" in ptype or ptype.split()[0] in handles:
                assert t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer), (name, p)
            else:
                base = " ".join(ptype.split()[:-1])
                want = scalars.get(base, ctypes.c_int)  # enums pass as int
                assert ctypes.sizeof(t) == ctypes.sizeof(want) and t != ctypes.c_void_p, (name, p)
        want_ret = {"srp_status": ctypes.c_int, "double": ctypes.c_double,
                    "const char*": ctypes.c_char_p, "void": None}[ret.split()[-1] if ret != "const char*" else ret]
        assert restype == want_ret, (name, ret, restype)
