"""GPU walker lists against the CPU oracle, element by element, after every
iteration: keys, int64 fixed-point populations and the cached diagonal bit for
bit; estimator records (exact 128-bit numerator, shift) bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1811_11679_gb300 import hande, inputs

pytestmark = pytest.mark.gpu
F = 2 ** 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _same_lists(g, c, it):
    kg, pg, hg, fg = g.walkers()
    kc, pc, hc, fc = c.walkers()
    assert kg.shape == kc.shape, f"iteration {it}: {len(kg)} vs {len(kc)} determinants"
    assert np.array_equal(kg, kc), f"iteration {it}: keys differ"
    assert np.array_equal(pg, pc), f"iteration {it}: populations differ"
    assert np.array_equal(hg.view(np.int64), hc.view(np.int64)), f"iteration {it}: diagonal differs"
    assert np.array_equal(fg & 1, fc & 1), f"iteration {it}: core flags differ"
    return len(kg)


def _same_records(g, c):
    eg = g.estimators()
    ec = c.records()
    n = len(ec["iter"])
    for k in ("iter", "nw_pre", "n0", "num_hi", "nw_post", "ndet", "natt", "nspawn"):
        assert np.array_equal(eg[k][-n:], ec[k]), k
    assert np.array_equal(eg["num_lo"][-n:], ec["num_lo"])
    assert np.array_equal(eg["shift"][-n:].view(np.int64), ec["shift"].view(np.int64))
    assert np.array_equal(eg["num"][-n:].view(np.int64), ec["num"].view(np.int64))
    return eg


def _run_parity(sysd, q, iters, every=1):
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    eg, kc = g.reference()
    assert eg == c.e_ref and np.array_equal(kc, c.reference())
    sizes = []
    done = 0
    while done < iters:
        step = min(every, iters - done)
        g.iterate(step)
        c.iterate(step)
        done += step
        sizes.append(_same_lists(g, c, done))
    _same_records(g, c)
    g.close()
    return sizes


def test_hubbard_ring_integer_walkers_every_iteration():
    """1D Hubbard ring, 8 sites, integer walkers: bit-exact for 400 iterations."""
    sysd, q = inputs.workload("hubbard8")
    sizes = _run_parity(sysd, q, 400)
    assert max(sizes) > 1000


def test_hubbard_full_run_2000_iterations():
    sysd, q = inputs.workload("hubbard8")
    _run_parity(sysd, q, 2000, every=250)


def test_ueg_128bit_initiator_real_weights():
    """UEG 14e / 38 orbitals (76 spin orbitals, two key words), initiator, real weights."""
    sysd, q = inputs.workload("ueg14", target_population=20000, init_pop=1000)
    sizes = _run_parity(sysd, q, 150)
    assert max(sizes) > 1000


@pytest.mark.parametrize("annihilation", [1, 2])
def test_ueg_512bit_keys(annihilation):
    """512-bit keys on block tiles and on the warp-per-bucket path (the default)."""
    sysd = inputs.ueg_system(14, 38, 1.0, key_words=8)
    q = inputs.qmc_params(tau=0.002, target_population=5000, initiator=1, real_amplitudes=1,
                          spawn_cutoff=0.1, init_pop=100, seed=7)
    q["annihilation"] = annihilation
    _run_parity(sysd, q, 80)


def test_ueg_128bit_block_annihilation():
    """128-bit keys on the block-tile annihilation (the default there is one warp per bucket)."""
    sysd, q = inputs.workload("ueg14", target_population=20000, init_pop=1000, annihilation=1)
    _run_parity(sysd, q, 60)


def test_ueg_64bit_keys_19_orbitals():
    sysd = inputs.ueg_system(14, 19, 2.0)
    assert sysd["key_words"] == 1
    q = inputs.qmc_params(tau=0.005, target_population=5000, initiator=1, real_amplitudes=1,
                          spawn_cutoff=0.1, init_pop=100, seed=11)
    _run_parity(sysd, q, 100)


def test_molecule_heat_bath_semistochastic():
    """Synthetic 28-orbital molecule: heat-bath generator, initiator, real weights,
    deterministic space of 300 chosen at iteration 40."""
    sysd, q = inputs.workload("molecule28", target_population=30000, semi_stoch_size=300,
                              semi_stoch_start=40)
    _run_parity(sysd, q, 120)


def test_deterministic_limit_against_oracle():
    """Whole-space core from a given list (start 0): exact projection on both sides."""
    import _brute as B
    dets, _ = B.hubbard_hamiltonian(6, 3, 3, 1.0, 4.0, True)
    rng = np.random.default_rng(1)
    keys = np.array([B.bits_to_words(d, 1) for d in dets], dtype=np.uint64)
    pops = (rng.integers(F // 10, F // 3, len(dets)) * rng.choice([-1, 1], len(dets))).astype(np.int64)
    sysd = inputs.hubbard_system(L=6, nalpha=3, nbeta=3)
    q = inputs.qmc_params(tau=0.05, target_population=0.5 * np.abs(pops).sum() / F, real_amplitudes=1,
                          spawn_cutoff=0.01, semi_stoch_size=len(dets), semi_stoch_start=0,
                          shift_damping=0.5, seed=3)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    g.set_walkers(keys, pops)
    c.set_walkers(keys, pops)
    for it in range(60):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
    _same_records(g, c)


def test_runs_are_deterministic_on_the_gpu():
    sysd, q = inputs.workload("ueg14", target_population=20000, init_pop=100)
    a = hande.Hande(sysd, q)
    b = hande.Hande(sysd, q)
    a.iterate(60)
    b.iterate(60)
    ka, pa, _, _ = a.walkers()
    kb, pb, _, _ = b.walkers()
    assert np.array_equal(ka, kb) and np.array_equal(pa, pb)


def test_spawn_capacity_overflow_reports_error():
    sysd, q = inputs.workload("hubbard8", spawn_capacity=64)
    g = hande.Hande(sysd, q)
    g.iterate(5)
    with pytest.raises(hande.HandeError) as e:
        g.synchronize()
    assert e.value.status == -3
    with pytest.raises(hande.HandeError) as e:
        g.iterate(1)
    assert e.value.status == -7


def test_state_capacity_overflow_reports_error():
    sysd, q = inputs.workload("ueg14", target_population=1e6, init_pop=500, state_capacity=300)
    g = hande.Hande(sysd, q)
    g.iterate(30)
    with pytest.raises(hande.HandeError) as e:
        g.estimators()
    assert e.value.status == -3


def test_set_get_walkers_roundtrip_and_validation():
    sysd, q = inputs.workload("ueg14", target_population=20000, init_pop=100)
    g = hande.Hande(sysd, q)
    g.iterate(20)
    k, p, h, f = g.walkers()
    g2 = hande.Hande(sysd, q)
    g2.set_walkers(k, p)
    k2, p2, h2, _ = g2.walkers()
    assert np.array_equal(k, k2) and np.array_equal(p, p2)
    assert np.array_equal(h.view(np.int64), h2.view(np.int64))   # diagonal recomputed on the device
    with pytest.raises(hande.HandeError):
        g2.set_walkers(k[::-1].copy(), p[::-1].copy())             # not ascending
    _, ref = g2.reference()
    other = [i for i in range(len(k)) if not np.array_equal(k[i], ref)][:1]
    with pytest.raises(hande.HandeError):
        g2.set_walkers(k[other].copy(), p[other].copy())           # reference missing
    bad = k.copy()
    bad[0, 0] ^= np.uint64(1)                                      # wrong electron number
    with pytest.raises(hande.HandeError):
        g2.set_walkers(bad, p)


@pytest.mark.parametrize("annihilation,tile", [(1, 64), (1, 256), (2, 64)])
def test_oversized_buckets_small_tiles(annihilation, tile):
    """Small annihilation tiles force many buckets through the oversized paths
    (block tiles: spawn-sampled sub-ranges, two-pass merge; one warp per bucket:
    batches of new keys in key order); lists stay bit-identical."""
    # 64 x tile walkers on the reference (about one attempt in fifteen spawns
    # from it: most heat-bath draws land on occupied orbitals): the first
    # iteration's single bucket receives several times more spawns than the tile
    sysd, q = inputs.workload("molecule28", target_population=1e5, semi_stoch_size=200,
                              semi_stoch_start=30, tile_capacity=tile, annihilation=annihilation,
                              init_pop=64 * tile)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    seen = deferred = 0
    for it in range(80):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
        d = g.diagnostics()
        seen = max(seen, d["max_bucket_spawns"])
        deferred = max(deferred, d["deferred_buckets"])
    _same_records(g, c)
    assert seen > tile            # some bucket held more spawns than the tile
    if annihilation == 2:
        assert deferred > 0       # the warp path handed buckets to block tiles


@pytest.mark.parametrize("annihilation", [1, 2])
def test_oversized_bucket_single_bucket_start(annihilation):
    """3000 walkers on the reference and a one-determinant list: the first
    iteration puts every spawn in one bucket, far above a 64-key tile."""
    sysd, q = inputs.workload("molecule28", target_population=1e5, init_pop=3000, tile_capacity=64,
                              annihilation=annihilation)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    g.iterate(1)
    c.iterate(1)
    d = g.diagnostics()
    assert d["max_bucket_spawns"] > 64
    if annihilation == 2:
        assert d["deferred_buckets"] > 0   # the warp path handed the bucket to block tiles
    _same_lists(g, c, 1)
    for it in range(1, 30):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
    _same_records(g, c)


@pytest.mark.parametrize("annihilation", [1, 2])
def test_oversized_buckets_from_synthetic_start(annihilation):
    """A synthetic list whose spawn keys are skewed against the main-list
    splitters (the benchmark's starting state, scaled down)."""
    sysd, q = inputs.workload("molecule28", target_population=2e5, semi_stoch_size=500, semi_stoch_start=0,
                              tile_capacity=64, annihilation=annihilation)
    keys, pops = inputs.synthetic_walkers(sysd, 40000, 2e5)
    g = hande.Hande(sysd, q)
    c = oracle.Oracle(sysd, q)
    g.set_walkers(keys, pops)
    c.set_walkers(keys, pops)
    seen = 0
    for it in range(8):
        g.iterate(1)
        c.iterate(1)
        _same_lists(g, c, it + 1)
        seen = max(seen, g.diagnostics()["max_bucket_spawns"])
    _same_records(g, c)
    assert seen > 64              # buckets beyond a 64-key tile occurred


def test_hubbard_2d_tilted_8_site_integer_walkers():
    """2D Hubbard model on the tilted 8-site cluster (lattice vectors (2, 2),
    (2, -2)), integer walkers: bit-exact for 300 iterations."""
    sysd = inputs.hubbard_lattice_system([[2, 2], [2, -2]], 4, 4, t=1.0, U=4.0)
    q = inputs.qmc_params(tau=0.01, target_population=3000, seed=4)
    sizes = _run_parity(sysd, q, 300)
    assert max(sizes) > 500


def test_hubbard18_2d_semistochastic():
    """The half-filled 18-site cluster at U/t = 1.3 (the paper's semi-stochastic
    example), initiator, real weights, a 500-determinant deterministic space
    chosen at iteration 60."""
    sysd, q = inputs.workload("hubbard18_2d", target_population=20000, semi_stoch_size=500, semi_stoch_start=60)
    sizes = _run_parity(sysd, q, 120)
    assert max(sizes) > 2000
