"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and exports every
function that include/ots.h declares; the binding's structures match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ots.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ots_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ots_create_problem", "ots_sinkhorn_solve", "ots_get_flows", "ots_get_duals",
              "ots_destroy_problem", "ots_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2106_14485_gb300 import build, ots
    build.build()
    lib = ots.load_library()
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) == set(ots.EXPORTED)


def test_status_strings_need_no_gpu():
    from paper_2106_14485_gb300 import ots
    assert ots.ots_status_string(0) == "OTS_OK"
    assert ots.ots_status_string(2) == "OTS_ERR_INFEASIBLE"
    assert ots.ots_status_string(ots.OTS_PENDING) == "OTS_PENDING"
    o = ots.ots_default_solve_opts()
    assert o.tol == 1e-6 and o.max_iters == 100000 and o.check_every == 10 and o.use_graph == 1


def test_struct_layout_matches_header():
    """Compile a tiny C program against ots.h that prints sizeof/offsetof and compare."""
    import subprocess
    import tempfile
    from paper_2106_14485_gb300 import ots
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "ots.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(ots_problem_desc), offsetof(ots_problem_desc, eps),
         offsetof(ots_problem_desc, stream), offsetof(ots_problem_desc, alloc_ctx));
  printf("%zu %zu\n", sizeof(ots_solve_opts), offsetof(ots_solve_opts, threads_per_node));
  printf("%zu %zu\n", sizeof(ots_solve_report), offsetof(ots_solve_report, status));
  printf("%zu %zu %zu\n", sizeof(ots_batch_desc), offsetof(ots_batch_desc, ticks_per_launch),
         offsetof(ots_batch_desc, alloc_ctx));
  printf("%zu %zu\n", sizeof(ots_batch_stats), offsetof(ots_batch_stats, d2h_bytes));
  printf("%d\n", (int)OTS_PENDING);
  printf("%zu %zu %zu\n", sizeof(ots_server_desc), offsetof(ots_server_desc, mode),
         sizeof(ots_server_stats));
  printf("%zu\n", offsetof(ots_server_stats, batch_ticks));
  printf("%zu %zu\n", sizeof(ots_linear_stats), offsetof(ots_linear_stats, kernel_ms));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    vals = list(map(int, out))
    D, O, R = ots.ProblemDesc, ots.SolveOpts, ots.SolveReport
    assert vals[0] == ctypes.sizeof(D) and vals[1] == D.eps.offset
    assert vals[2] == D.stream.offset and vals[3] == D.alloc_ctx.offset
    assert vals[4] == ctypes.sizeof(O) and vals[5] == O.threads_per_node.offset
    assert vals[6] == ctypes.sizeof(R) and vals[7] == R.status.offset
    B, BS = ots.BatchDesc, ots.BatchStats
    assert vals[8] == ctypes.sizeof(B) and vals[9] == B.ticks_per_launch.offset and vals[10] == B.alloc_ctx.offset
    assert vals[11] == ctypes.sizeof(BS) and vals[12] == BS.d2h_bytes.offset
    assert vals[13] == ots.OTS_PENDING
    SD, SS = ots.ServerDesc, ots.ServerStats
    assert vals[14] == ctypes.sizeof(SD) and vals[15] == SD.mode.offset and vals[16] == ctypes.sizeof(SS)
    assert vals[17] == SS.batch_ticks.offset
    LS = ots.LinearStats
    assert vals[18] == ctypes.sizeof(LS) and vals[19] == LS.kernel_ms.offset


def test_oracle_is_not_imported_by_the_product():
    """The product path never loads the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2106_14485_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f
                assert "libots_oracle" not in txt and "ots_oracle" not in txt, f


def test_time_varying_costs_are_validated_on_the_host():
    """Rejected before any device work: wrong combination and invalid values."""
    import numpy as np
    from paper_2106_14485_gb300 import instances as I, ots
    inst = I.rgg_instance(seed=3, n=30, L=2, T=6, eps=0.1)
    inst.state_cost_t = np.ones((inst.T - 2, inst.n_states))
    inst.commodity_cost = np.ones((inst.L, inst.n_states))
    with pytest.raises(ots.OTSError) as e:
        ots.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == ots.OTS_ERR_INVALID_ARG
    inst.commodity_cost = None
    inst.state_cost_t[1, 3] = np.nan
    with pytest.raises(ots.OTSError) as e:
        ots.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == ots.OTS_ERR_INVALID_ARG


def test_per_interval_capacities_are_validated_on_the_host():
    import numpy as np
    from paper_2106_14485_gb300 import instances as I, ots
    inst = I.rgg_instance(seed=3, n=30, L=2, T=6, eps=0.1)
    inst.state_capacity_t = np.full((inst.T - 2, inst.n_states), np.inf)
    inst.state_capacity_t[2, 5] = -1.0
    with pytest.raises(ots.OTSError) as e:
        ots.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == ots.OTS_ERR_INVALID_ARG
    inst.state_capacity_t[2, 5] = np.nan
    with pytest.raises(ots.OTSError) as e:
        ots.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == ots.OTS_ERR_INVALID_ARG


def test_commodity_windows_are_validated_on_the_host():
    import numpy as np
    from paper_2106_14485_gb300 import instances as I, ots
    inst = I.rgg_instance(seed=3, n=30, L=2, T=6, eps=0.1)
    inst.commodity_t_in = np.array([1, 4], np.int32)
    inst.commodity_t_out = np.array([6, 4], np.int32)          # t_out <= t_in
    with pytest.raises(ots.OTSError) as e:
        ots.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == ots.OTS_ERR_INVALID_ARG
    inst.commodity_t_out = np.array([6, 6], np.int32)
    with pytest.raises(ots.OTSError) as e:                      # windows need every Psi_t kept
        ots.ots_create_problem(inst, allocator="cuda", psi_stride=3)
    assert e.value.code == ots.OTS_ERR_INVALID_ARG


def build_c_example():
    """Compile the plain-C example against include/ots.h and link it to libots.so."""
    import subprocess
    from paper_2106_14485_gb300 import build
    lib = build.build()
    pkg = os.path.dirname(lib)
    exe = os.path.join(pkg, "_build", "solve_grid")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(pkg, "examples", "solve_grid.c"), "-o", exe, "-L", pkg, "-lots",
                           "-Wl,-rpath," + pkg, "-lm"])
    return exe


def test_c_example_builds_against_the_header_and_the_library():
    assert os.path.exists(build_c_example())


def test_c_program_checks_a_descriptor_without_a_gpu():
    """A plain C caller validates descriptors through the ABI on a machine without a GPU: a 3-node
    line with one commodity is accepted; an unreachable sink and a negative capacity are refused
    with their status codes."""
    import subprocess
    import tempfile
    from paper_2106_14485_gb300 import build
    pkg = os.path.dirname(build.build())
    prog = r'''
#include <math.h>
#include <stdio.h>
#include "ots.h"
int main(void) {
  int32_t src[4] = {0, 1, 1, 2}, dst[4] = {1, 2, 0, 1};
  double cost[4] = {1, 1, 1, 1}, cap[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  int32_t comm[1] = {0}, s_state[1] = {4 + 0}, z_state[1] = {4 + 2};
  double mass[1] = {1.0};
  ots_problem_desc d = {0};
  d.n_nodes = 3; d.n_edges = 4; d.edge_src = src; d.edge_dst = dst; d.edge_cost = cost; d.edge_capacity = cap;
  d.add_wait_loops = 1; d.T = 4; d.L = 1; d.eps = 0.1;
  d.n_sources = 1; d.src_commodity = comm; d.src_state = s_state; d.src_mass = mass;
  d.n_sinks = 1; d.snk_commodity = comm; d.snk_state = z_state; d.snk_mass = mass;
  printf("%d\n", (int)ots_check_problem(&d));
  d.T = 3;                       /* wait loop, two streets, wait loop: three transitions > T - 1 */
  printf("%d\n", (int)ots_check_problem(&d));
  d.T = 4; cap[1] = -1.0;
  printf("%d %s\n", (int)ots_check_problem(&d), ots_last_error());
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "check.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "check")
        subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), c, "-o", exe,
                               "-L", pkg, "-lots", "-Wl,-rpath," + pkg])
        out = subprocess.check_output([exe]).decode().split("\n")
    from paper_2106_14485_gb300 import ots
    assert int(out[0]) == ots.OTS_OK
    assert int(out[1]) == ots.OTS_ERR_INFEASIBLE
    assert int(out[2].split()[0]) == ots.OTS_ERR_INVALID_ARG and "capacity" in out[2]
