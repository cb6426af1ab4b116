"""Host-side validation of ots_create_problem (no GPU needed): every malformed descriptor is
rejected with its status code before any device work.  The rules are the problem statement of
Section 3.2 (eq. multicommodity: positive source and sink masses, equal per commodity; capacities
d >= 0; eps > 0; T >= 3 because Algorithm 2 needs hatPsi_2 and Psi_{T-1}) and the reachability of
every sink from its commodity's sources within T - 1 transitions (Section 3.1)."""
import numpy as np
import pytest

from paper_2106_14485_gb300 import instances as I


@pytest.fixture(scope="module")
def O():
    from paper_2106_14485_gb300 import build, ots
    build.build()
    ots.load_library()
    return ots


def base():
    return I.rgg_instance(seed=3, n=30, L=2, T=6, eps=0.1)


def copy(inst):
    return I.Instance(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in inst.__dict__.items()})


def _eps_zero(x): x.eps = 0.0
def _eps_nan(x): x.eps = float("nan")
def _eps_inf(x): x.eps = float("inf")
def _t_two(x): x.T = 2
def _neg_mass(x): x.src_mass[0] = -x.src_mass[0]
def _inf_mass(x): x.src_mass[0] = np.inf
def _zero_mass(x): x.snk_mass[0] = 0.0
def _unequal_mass(x): x.snk_mass = x.snk_mass * 1.5
def _state_range(x): x.src_state[0] = x.n_states
def _state_negative(x): x.snk_state[0] = -1
def _comm_range(x): x.src_comm[0] = x.L
def _edge_range(x): x.edge_dst[0] = x.n_nodes
def _cost_nan(x): x.edge_cost[0] = np.nan
def _cost_inf(x): x.edge_cost[0] = np.inf
def _cap_negative(x): x.edge_cap[0] = -0.5
def _cap_nan(x): x.edge_cap[0] = np.nan
def _commodity_cost_inf(x):
    x.commodity_cost = np.ones((x.L, x.n_states)); x.commodity_cost[1, 2] = np.inf
def _commodity_capacity_negative(x):
    x.commodity_capacity = np.full((x.L, x.n_states), np.inf); x.commodity_capacity[0, 4] = -1.0
def _no_sink_for_commodity(x):
    keep = x.snk_comm != 1
    x.snk_comm, x.snk_state, x.snk_mass = x.snk_comm[keep], x.snk_state[keep], x.snk_mass[keep]
def _windows_outside(x):
    x.commodity_t_in = np.array([0, 1], np.int32); x.commodity_t_out = np.array([x.T, x.T], np.int32)


CASES = [_eps_zero, _eps_nan, _eps_inf, _t_two, _neg_mass, _inf_mass, _zero_mass, _unequal_mass, _state_range,
         _state_negative, _comm_range, _edge_range, _cost_nan, _cost_inf, _cap_negative, _cap_nan,
         _commodity_cost_inf, _commodity_capacity_negative, _no_sink_for_commodity, _windows_outside]


@pytest.mark.parametrize("mutate", CASES, ids=[c.__name__.strip("_") for c in CASES])
def test_malformed_descriptor_is_rejected(O, mutate):
    inst = copy(base())
    mutate(inst)
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == O.OTS_ERR_INVALID_ARG, e.value
    with pytest.raises(O.OTSError) as e:                          # the same through the host-only check
        O.ots_check_problem(inst)
    assert e.value.code == O.OTS_ERR_INVALID_ARG, e.value


def test_negative_psi_stride_is_rejected(O):
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(base(), allocator="cuda", psi_stride=-1)
    assert e.value.code == O.OTS_ERR_INVALID_ARG


def test_sink_out_of_reach_is_infeasible(O):
    """Opposite corners of a 5x5 grid are 8 moves apart: with T = 5 (4 transitions) the sink cannot
    be reached, which the host search reports before any device work."""
    inst = I.grid_single_commodity(0, T=5)
    E = inst.n_edges
    inst.src_comm = np.zeros(1, np.int32); inst.src_state = np.array([E + 0], np.int32); inst.src_mass = np.array([1.0])
    inst.snk_comm = np.zeros(1, np.int32); inst.snk_state = np.array([E + 24], np.int32); inst.snk_mass = np.array([1.0])
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(inst, allocator="cuda")
    assert e.value.code == O.OTS_ERR_INFEASIBLE


def test_error_message_names_the_problem(O):
    inst = copy(base())
    inst.edge_cap[3] = -2.0
    with pytest.raises(O.OTSError) as e:
        O.ots_create_problem(inst, allocator="cuda")
    assert "capacity" in str(e.value)


def _valid_instances():
    yield I.grid_single_commodity(0)
    yield I.rgg400(0)
    yield I.traffic_grid(0)                                       # the benchmark workload (host part only)
    yield I.with_time_varying_costs(I.rgg_instance(seed=3, n=60, L=5, T=12, eps=0.05), seed=1, closures=3)
    yield I.with_time_varying_capacities(I.rgg_instance(seed=3, n=60, L=5, T=12, eps=0.05), seed=1)
    yield I.with_commodity_windows(I.rgg_instance(seed=3, n=60, L=5, T=14, eps=0.05), seed=2)
    yield I.single_commodity_instance(0)
    x = I.rgg_instance(seed=3, n=40, L=3, T=10, eps=0.05)
    x.commodity_capacity = np.full((x.L, x.n_states), 0.5)
    yield x


def test_valid_instances_pass_the_host_checks(O):
    """The host part of the construction (state graph, per-state data, boundary triples,
    reachability) accepts every workload the tests and the benchmark use, without a device."""
    for inst in _valid_instances():
        O.ots_check_problem(inst)


def test_host_check_reports_unreachable_sinks(O):
    inst = I.grid_single_commodity(0, T=5)
    E = inst.n_edges
    inst.src_comm = np.zeros(1, np.int32); inst.src_state = np.array([E + 0], np.int32); inst.src_mass = np.array([1.0])
    inst.snk_comm = np.zeros(1, np.int32); inst.snk_state = np.array([E + 24], np.int32); inst.snk_mass = np.array([1.0])
    with pytest.raises(O.OTSError) as e:
        O.ots_check_problem(inst)
    assert e.value.code == O.OTS_ERR_INFEASIBLE
    inst.T = 9            # wait loop, 8 streets, wait loop: 9 transitions, one more than T - 1 = 8
    with pytest.raises(O.OTSError) as e:
        O.ots_check_problem(inst)
    assert e.value.code == O.OTS_ERR_INFEASIBLE
    inst.T = 10
    O.ots_check_problem(inst)


def test_commodity_count_limits(O):
    """The ABI takes 1 <= L <= 4096 (at most 256 threads per node row with four chunks of four
    commodities); the host part accepts both ends and rejects one more."""
    for L in (1, 4096):
        O.ots_check_problem(I.rgg_instance(seed=3, n=30, L=L, T=6, eps=0.1))
    x = I.rgg_instance(seed=3, n=30, L=4097, T=6, eps=0.1)
    with pytest.raises(O.OTSError) as e:
        O.ots_check_problem(x)
    assert e.value.code == O.OTS_ERR_INVALID_ARG


def test_explicit_state_graph_is_validated_on_the_host():
    """ots_check_problem on explicit state graphs (no device): the traffic-routing model passes;
    a tail out of range or a storage flag other than 0 / 1 is an invalid argument; a sink that
    no exact walk of T-1 transitions reaches is infeasible."""
    from paper_2106_14485_gb300 import ots
    ots.load_library()
    good = I.traffic_routing_instance(seed=1, rows=4, cols=4, L=3, T=9, eps=0.1)
    ots.ots_check_problem(good)
    bad = I.traffic_routing_instance(seed=1, rows=4, cols=4, L=3, T=9, eps=0.1)
    bad.state_tail = bad.state_tail.copy()
    bad.state_tail[0] = bad.n_nodes
    with pytest.raises(ots.OTSError) as e:
        ots.ots_check_problem(bad)
    assert e.value.code == ots.OTS_ERR_INVALID_ARG
    bad = I.traffic_routing_instance(seed=1, rows=4, cols=4, L=3, T=9, eps=0.1)
    bad.state_hold = bad.state_hold.copy()
    bad.state_hold[0] = 2
    with pytest.raises(ots.OTSError) as e:
        ots.ots_check_problem(bad)
    assert e.value.code == ots.OTS_ERR_INVALID_ARG
    short = I.traffic_routing_instance(seed=1, rows=4, cols=4, L=3, T=9, eps=0.1)
    short.T = 3                                    # two transitions cannot cross the grid
    with pytest.raises(ots.OTSError) as e:
        ots.ots_check_problem(short)
    assert e.value.code == ots.OTS_ERR_INFEASIBLE
