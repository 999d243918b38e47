"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point the header declares, the ctypes structures match the C
layout, and argument validation rejects bad calls before any launch."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2603_23343_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbpcg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbpcg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return B.load()


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in gbpcg.h but not exported"
    assert sorted(B.EXPORTS) == sorted(names)


def test_version_string(lib):
    assert B.version().startswith("gbpcg") and "sm_103a" in B.version()


def test_struct_layout_matches_header(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gbpcg.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu %zu\\n", sizeof(gbpcg_grid), offsetof(gbpcg_grid, k_block), offsetof(gbpcg_grid, kbx), offsetof(gbpcg_grid, kbz));\n'
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(gbpcg_opts), offsetof(gbpcg_opts, flags), offsetof(gbpcg_opts, workspace), offsetof(gbpcg_opts, workspace_bytes), offsetof(gbpcg_opts, max_outer));\n'
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(gbpcg_result), offsetof(gbpcg_result, rel_res_recursive), offsetof(gbpcg_result, time_ms), offsetof(gbpcg_result, pass_launches), offsetof(gbpcg_result, replacements));\n'
        " return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.dirname(HEADER)}", str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    g = [int(v) for v in out[0].split()]
    o = [int(v) for v in out[1].split()]
    r = [int(v) for v in out[2].split()]
    assert g == [ctypes.sizeof(B.Grid), B.Grid.k_block.offset, B.Grid.kbx.offset, B.Grid.kbz.offset]
    assert o == [ctypes.sizeof(B.Opts), B.Opts.flags.offset, B.Opts.workspace.offset, B.Opts.workspace_bytes.offset,
                 B.Opts.max_outer.offset]
    assert r == [ctypes.sizeof(B.Result), B.Result.rel_res_recursive.offset, B.Result.time_ms.offset,
                 B.Result.pass_launches.offset, B.Result.replacements.offset]


def test_tile_configs_enumerate(lib):
    cfgs = B.tile_configs()
    assert len(cfgs) == 10 and cfgs[0] == (64, 16, 4) and cfgs[6] == (256, 4, 4) and cfgs[9] == (256, 4, 3)
    for tx, ty, st in cfgs:
        assert tx % 4 == 0 and ty >= 1 and st >= 2
    g = _grid(16, 16, 16)
    n = ctypes.c_size_t(0)
    o = B.make_opts(tile_cfg=B.tile_cfg_code(len(cfgs) - 1, 0))
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.OK
    o = B.make_opts(tile_cfg=B.tile_cfg_code(len(cfgs), 0))
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG


def test_workspace_size_is_host_logic(lib):
    n = 64 * 48 * 40
    ws = B.workspace_size((40, 48, 64))
    assert ws >= 3 * 4 * n  # z and two p buffers in FP32
    ws_io = B.workspace_size((40, 48, 64), host_io=True)
    assert ws_io >= ws + 2 * 4 * n


def _grid(nx, ny, nz):
    return B.Grid(nx, ny, nz, None, 1, 1, 1)


@pytest.mark.parametrize("dims", [(0, 4, 4), (4, -1, 4), (4, 4, 0)])
def test_bad_grid_is_rejected_before_launch(lib, dims):
    g = _grid(*dims)
    rc = lib.gbpcg_stencil_apply(ctypes.byref(g), B.F32, ctypes.c_void_p(16), ctypes.c_void_p(32), None)
    assert rc == B.ERR_ARG
    assert "invalid argument" in B.last_error()


def test_bad_dtype_and_aliasing_rejected(lib):
    g = _grid(8, 8, 8)
    assert lib.gbpcg_stencil_apply(ctypes.byref(g), 7, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == B.ERR_ARG
    assert lib.gbpcg_stencil_apply(ctypes.byref(g), B.F32, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == B.ERR_ARG
    assert lib.gbpcg_stencil_apply(ctypes.byref(g), B.F32, None, ctypes.c_void_p(16), None) == B.ERR_ARG


def test_block_coefficient_needs_block_edges(lib):
    g = B.Grid(8, 8, 8, 4096, 0, 8, 8)
    assert lib.gbpcg_stencil_apply(ctypes.byref(g), B.F32, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == B.ERR_ARG


def test_dot_argument_checks(lib):
    small = ctypes.c_size_t(16)
    rc = lib.gbpcg_dot(10, B.F32, ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(64),
                       ctypes.c_void_p(256), small, None)
    assert rc == B.ERR_ARG and "workspace" in B.last_error()
    rc = lib.gbpcg_dot(-1, B.F32, None, None, ctypes.c_void_p(64), ctypes.c_void_p(256),
                       B.dot_workspace_size(), None)
    assert rc == B.ERR_ARG
    rc = lib.gbpcg_dot(10, B.F32, ctypes.c_void_p(16), ctypes.c_void_p(32), None, ctypes.c_void_p(256),
                       B.dot_workspace_size(), None)
    assert rc == B.ERR_ARG


def test_dot_noalloc_rejects_n_beyond_its_static_scratch(lib):
    # checked before any CUDA call: n above 2^30 does not fit the static partial-sum array
    rc = lib.gbpcg_dot_noalloc((1 << 30) + 1, B.F32, ctypes.c_void_p(16), ctypes.c_void_p(32),
                               ctypes.c_void_p(64), None)
    assert rc == B.ERR_ARG and "static scratch" in B.last_error()
    assert lib.gbpcg_dot_noalloc(-1, B.F32, None, None, ctypes.c_void_p(64), None) == B.ERR_ARG


def test_axpy_argument_checks(lib):
    assert lib.gbpcg_axpy(-5, B.F32, 1.0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == B.ERR_ARG
    assert lib.gbpcg_axpy(5, B.F32, 1.0, None, ctypes.c_void_p(32), None) == B.ERR_ARG
    assert lib.gbpcg_axpy(0, B.F32, 1.0, None, None, None) == B.OK  # empty is a no-op


def test_solve_argument_checks(lib):
    g = _grid(16, 16, 16)
    o = B.make_opts()
    r = B.Result()
    # no workspace
    rc = lib.gbpcg_pcg_solve(ctypes.byref(g), ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.byref(o),
                             ctypes.byref(r), None)
    assert rc == B.ERR_ARG and "workspace" in B.last_error()
    o.tol = -1.0
    n = ctypes.c_size_t(0)
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    o = B.make_opts(storage=5)
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    # 16-bit storage means iterative refinement: FP64 b/x and a sane inner tolerance
    o = B.make_opts(storage=B.BF16, io_dtype=B.F32)
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    o = B.make_opts(storage=B.F16, io_dtype=B.F64, inner_tol=1.5)
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    o = B.make_opts(storage=B.F16, io_dtype=B.F64)
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.OK
    assert n.value >= 16 ** 3 * (4 + 4 + 4 * 2)


def test_batched_argument_checks(lib):
    grids = (B.Grid * 2)(_grid(16, 16, 16), _grid(32, 8, 8))
    n = ctypes.c_size_t(0)
    o = B.make_opts()
    assert lib.gbpcg_workspace_size_batched(2, grids, ctypes.byref(o), ctypes.byref(n)) == B.OK
    single = ctypes.c_size_t(0)
    total = 0
    for i in range(2):
        assert lib.gbpcg_workspace_size(ctypes.byref(grids[i]), ctypes.byref(o), ctypes.byref(single)) == B.OK
        total += single.value
    assert n.value >= total
    ot = B.make_opts(autotune=True)
    nt = ctypes.c_size_t(0)
    assert lib.gbpcg_workspace_size_batched(2, grids, ctypes.byref(ot), ctypes.byref(nt)) == B.OK
    assert nt.value >= n.value + 4 * (16 ** 3 + 32 * 64)
    assert lib.gbpcg_workspace_size_batched(0, grids, ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    ob = B.make_opts(storage=B.BF16, io_dtype=B.F64)
    assert lib.gbpcg_workspace_size_batched(2, grids, ctypes.byref(ob), ctypes.byref(n)) == B.ERR_ARG
    oh = B.make_opts(host_io=True)
    assert lib.gbpcg_workspace_size_batched(2, grids, ctypes.byref(oh), ctypes.byref(n)) == B.ERR_ARG
    r = (B.Result * 2)()
    assert lib.gbpcg_pcg_solve_batched(2, grids, None, None, ctypes.byref(o), r, None) == B.ERR_ARG


def test_autotune_record_checks(lib):
    g = _grid(300, 8, 8)
    o = B.make_opts()
    assert lib.gbpcg_autotune_record(ctypes.byref(g), ctypes.byref(o), 0) == B.ERR_ARG
    assert lib.gbpcg_autotune_record(ctypes.byref(g), ctypes.byref(o), B.tile_cfg_code(6, 6)) == B.ERR_ARG
    assert lib.gbpcg_autotune_record(ctypes.byref(g), ctypes.byref(o), B.tile_cfg_code(2, 2)) == B.OK


def test_last_error_is_cleared_on_success(lib):
    g = _grid(0, 1, 1)
    lib.gbpcg_stencil_apply(ctypes.byref(g), B.F32, None, None, None)
    assert B.last_error() != ""
    n = ctypes.c_size_t(0)
    g2 = _grid(4, 4, 4)
    o = B.make_opts()
    assert lib.gbpcg_workspace_size(ctypes.byref(g2), ctypes.byref(o), ctypes.byref(n)) == B.OK
    assert B.last_error() == ""


def test_learned_preconditioner_argument_checks(lib):
    n = ctypes.c_size_t(0)
    # every level must split into 128-voxel tiles of whole rows or planes
    assert lib.gbpcg_nn_workspace_size(30, 30, 30, 0, ctypes.byref(n)) == B.ERR_ARG
    assert lib.gbpcg_nn_workspace_size(32, 32, 32, 0, ctypes.byref(n)) == B.OK
    inference = n.value
    assert inference >= 32 ** 3 * (2 + 16 + 48 + 16) * 2  # finest-level BF16 activations
    assert lib.gbpcg_nn_workspace_size(32, 32, 32, 1, ctypes.byref(n)) == B.OK
    assert n.value > inference  # training adds the gradient buffers
    assert lib.gbpcg_conv3_workspace_size(8, 8, 8, 16, 16, ctypes.byref(n)) == B.OK
    ws_ok = n.value
    P = ctypes.c_void_p
    assert lib.gbpcg_conv3_forward(8, 8, 8, 16, 16, None, None, None, 0, None, 0, None) == B.ERR_ARG
    # 16-byte alignment of the arrays, 256-byte alignment and size of the workspace
    assert lib.gbpcg_conv3_forward(8, 8, 8, 16, 16, P(8), P(16), P(32), 0, P(256), ws_ok, None) == B.ERR_ARG
    assert lib.gbpcg_conv3_forward(8, 8, 8, 16, 16, P(16), P(32), P(48), 0, P(256), 16, None) == B.ERR_ARG
    assert lib.gbpcg_conv3_forward(8, 8, 8, 16, 16, P(16), P(32), P(48), 0, P(272), ws_ok, None) == B.ERR_ARG
    # no kernel for 24 output channels, or for a 3-channel weight gradient
    assert lib.gbpcg_conv3_workspace_size(8, 8, 8, 16, 24, ctypes.byref(n)) == B.OK
    assert lib.gbpcg_conv3_forward(8, 8, 8, 16, 24, P(16), P(32), P(48), 0, P(256), n.value, None) == B.ERR_ARG
    assert lib.gbpcg_conv3_workspace_size(8, 8, 8, 3, 16, ctypes.byref(n)) == B.OK
    assert lib.gbpcg_conv3_backward_weight(8, 8, 8, 3, 16, P(16), P(32), P(48), P(256), n.value, None) == B.ERR_ARG
    assert lib.gbpcg_nn_adam(-1, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, None) == B.ERR_ARG
    assert lib.gbpcg_nn_adam(10, None, None, None, None, 0, 1e-3, 0.9, 0.999, 1e-8, None) == B.ERR_ARG
    assert lib.gbpcg_nn_adam(0, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, None) == B.OK
    assert lib.gbpcg_nn_status(None, None) == B.ERR_ARG
    g = _grid(32, 32, 32)
    assert lib.gbpcg_nn_forward(ctypes.byref(g), None, None, None, P(256), inference, None) == B.ERR_ARG


def test_mode_flags_and_variant_argument_checks(lib):
    g = _grid(32, 32, 32)
    n = ctypes.c_size_t(0)
    o = B.make_opts(mode="split")
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.OK
    assert n.value >= 4 * 32 ** 3 * 4  # r, z, p, q
    for bad in (B.make_opts(mode="split", io_dtype=B.F64), B.make_opts(mode="host_loop", profile=True),
                B.make_opts(mode="host_loop", storage=B.BF16, io_dtype=B.F64)):
        assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(bad), ctypes.byref(n)) == B.ERR_ARG
    o = B.make_opts(mode="split")
    o.flags |= B.FLAG_HOST_LOOP
    assert lib.gbpcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    P = ctypes.c_void_p
    wsz = lib.gbpcg_dot_variant_workspace_size()
    assert wsz > 0
    assert lib.gbpcg_dot_variant(5, 16, P(256), P(512), P(768), P(1024), wsz, None) == B.ERR_ARG
    assert lib.gbpcg_dot_variant(0, 0, P(256), P(512), P(768), P(1024), wsz, None) == B.ERR_ARG
    assert lib.gbpcg_dot_variant(0, 16, P(260), P(512), P(768), P(1024), wsz, None) == B.ERR_ARG
    assert lib.gbpcg_dot_variant(0, 16, P(256), P(512), P(768), P(1024), wsz - 1, None) == B.ERR_ARG
    assert lib.gbpcg_stencil_apply_variant(ctypes.byref(g), 3, P(256), P(512), None) == B.ERR_ARG
    assert lib.gbpcg_stencil_apply_variant(ctypes.byref(g), 0, P(256), P(256), None) == B.ERR_ARG
    assert lib.gbpcg_stencil_apply_variant(ctypes.byref(g), 0, P(260), P(512), None) == B.ERR_ARG


def test_nn_tensor_info_is_host_logic(lib):
    """Every tensor the network leaves in a workspace lies inside it, inference workspaces refuse
    the training-only gradient tensors, and distinct tensors do not overlap."""
    n = ctypes.c_size_t(0)
    shape = (16, 16, 128)
    spans = []
    for training in (0, 1):
        assert lib.gbpcg_nn_workspace_size(128, 16, 16, training, ctypes.byref(n)) == B.OK
        total = n.value
        for i, name in enumerate(B.NN_TENSORS):
            off, dt, ch, lv = ctypes.c_size_t(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
            rc = lib.gbpcg_nn_tensor_info(128, 16, 16, training, i, ctypes.byref(off), ctypes.byref(dt),
                                          ctypes.byref(ch), ctypes.byref(lv))
            if i >= B.NN_TENSORS.index("gout") and not training:
                assert rc == B.ERR_ARG, name
                continue
            assert rc == B.OK, name
            esize = {B.F32: 4, B.BF16: 2, B.F64: 8}[dt.value]
            vox = 1 if lv.value < 0 else (shape[0] >> lv.value) * (shape[1] >> lv.value) * (shape[2] >> lv.value)
            assert off.value % 256 == 0 or lv.value < 0, name
            assert off.value + vox * ch.value * esize <= total, name
            if training:
                spans.append((off.value, off.value + vox * ch.value * esize, name))
    spans.sort()
    for (a0, a1, na), (b0, b1, nb) in zip(spans, spans[1:]):
        assert a1 <= b0, (na, nb)
    off, dt, ch, lv = ctypes.c_size_t(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    assert lib.gbpcg_nn_tensor_info(128, 16, 16, 1, len(B.NN_TENSORS), ctypes.byref(off), ctypes.byref(dt),
                                    ctypes.byref(ch), ctypes.byref(lv)) == B.ERR_ARG
    assert lib.gbpcg_nn_tensor_info(30, 30, 30, 1, 0, ctypes.byref(off), ctypes.byref(dt), ctypes.byref(ch),
                                    ctypes.byref(lv)) == B.ERR_ARG


def test_fcg_argument_checks(lib):
    g = _grid(32, 32, 32)
    n = ctypes.c_size_t(0)
    o = B._fcg_opts(1e-6, 100)
    assert lib.gbpcg_fcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.OK
    default = n.value
    o.fcg_m = 1
    assert lib.gbpcg_fcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.OK
    # the default keeps 24 directions and their A-images: 46 more FP32 vectors than m = 1
    assert default - n.value >= 46 * 32 ** 3 * 4
    o.fcg_m = 33
    assert lib.gbpcg_fcg_workspace_size(ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    bad = [B.make_opts(io_dtype=B.F64)]  # Jacobi preconditioner: not this entry point
    for field, value in (("io_dtype", B.F32), ("storage", B.BF16), ("flags", B.FLAG_HOST_IO), ("tol", 0.0),
                         ("maxit", -1)):
        ob = B._fcg_opts(1e-6, 100)
        setattr(ob, field, value)
        bad.append(ob)
    for ob in bad:
        assert lib.gbpcg_fcg_workspace_size(ctypes.byref(g), ctypes.byref(ob), ctypes.byref(n)) == B.ERR_ARG
    g30 = _grid(30, 30, 30)
    assert lib.gbpcg_fcg_workspace_size(ctypes.byref(g30), ctypes.byref(o), ctypes.byref(n)) == B.ERR_ARG
    r = B.Result()
    o = B._fcg_opts(1e-6, 100)
    assert lib.gbpcg_fcg_solve(ctypes.byref(g), None, ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.byref(o),
                               ctypes.byref(r), None) == B.ERR_ARG
    assert lib.gbpcg_fcg_solve(ctypes.byref(g), ctypes.c_void_p(256), ctypes.c_void_p(264), ctypes.c_void_p(512),
                               ctypes.byref(o), ctypes.byref(r), None) == B.ERR_ARG  # b not 16-byte aligned
