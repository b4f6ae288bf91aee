"""The benchmark's roofline arithmetic on the headline plan's figures (N =
20480, near_nnz = 35,925,668, three far levels with L = 15, 10, 8, 1304 /
33,696 / 109,320 interaction-list entries, every element a source at every
level): the algorithmic bytes and operations are the ones written out by
hand (8 B per stored value + 16 B per element; 16 B per list entry and
direction, 2 L^2 directions; one sine and one cosine per element and
antipodal pair, L^2 pairs), and each fraction is achieved / peak."""
import bench

N, NNZ = 20480, 35925668
STATS = {"near_nnz": NNZ, "L": [15, 10, 8], "n_interactions": [1304, 33696, 109320],
         "n_src_elements": [N, N, N], "near_light_points": 86153328, "near_light_entries": 35477628,
         "near_heavy_points": 18631920, "near_heavy_entries": 448040}
KERNELS = {"k_near_spmv": {"total_ms": 64.9, "launches": 1020, "avg_us": 63.6},
           "k_aggregate": {"total_ms": 18.8, "launches": 1020, "avg_us": 18.4},
           "k_transfer": {"total_ms": 27.2, "launches": 1020, "avg_us": 26.6},
           "k_near_store": {"total_ms": 9.97, "launches": 20, "avg_us": 498.6},
           "k_near_store_heavy": {"total_ms": 1.75, "launches": 20, "avg_us": 87.4}}
PEAKS = {"hbm_gbs": 6662.6, "sm_max_mhz": 2070.0}


def test_dominant_kernel_roofline():
    r = bench.roofline(KERNELS, STATS, N, PEAKS, "measured")
    assert r["kernel"] == "k_near_spmv" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes"] == 8 * NNZ + 16 * N == 287733024
    assert abs(r["achieved"] - 287733024 / 63.6e-6 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 6662.6) < 1e-4
    assert r["peak"] == 6662.6


def test_traffic_record_only_for_the_captured_plan():
    # the stored DRAM traffic belongs to one near_nnz (and one kernel source)
    assert bench.spmv_traffic(NNZ + 2) is None
    # the kernel source and its forward launch are those of the capture (a
    # change to either nulls the record: take the ncu traffic again, then
    # update SPMV_TRAFFIC)
    assert bench.spmv_traffic(NNZ) == bench.SPMV_TRAFFIC["bytes"] == 291443712


def test_other_kernel_rooflines():
    out = bench.extra_rooflines(KERNELS, STATS, PEAKS)
    tr = out["k_transfer"]
    assert tr["bytes"] == (1304 * 450 + 33696 * 200 + 109320 * 128) * 16 == 341103360
    assert abs(tr["frac"] - tr["achieved"] / tr["peak"]) < 1e-4
    ag = out["k_aggregate"]
    assert ag["pair_terms"] == N * (225 + 100 + 64) == 7966720
    sfu = 152 * 16 * 2070e6 / 1e12
    assert abs(ag["peak"] - round(sfu, 3)) < 1e-9
    assert abs(ag["achieved"] - 2 * 7966720 / 18.4e-6 / 1e12) < 1e-3
    fp32 = 152 * 128 * 2 * 2070e6 / 1e12
    li = out["k_near_store_light"]
    assert li["flops_per_launch"] == 86153328 * bench.FLOPS_PER_POINT + 35477628 * bench.FLOPS_PER_ENTRY
    assert abs(li["peak"] - round(fp32, 1)) < 1e-9
    assert abs(li["frac"] - li["achieved"] / fp32) < 1e-3
