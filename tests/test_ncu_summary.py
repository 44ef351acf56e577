"""The Nsight Compute text summariser (no GPU): per-kernel launch counts,
totals and shares from an ncu launch list, with units converted and template
arguments kept; and the raw-page table of the roofline counters."""
import ncu_summary as S

HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",'
        '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(i, name, unit, value):
    return ('"%d","1","python3.12","host","%s","1","7","(256, 1, 1)","(1024, 1, 1)","0","10.3",'
            '"Command line profiler metrics","gpu__time_duration.sum","%s","%s"\n' % (i, name, unit, value))


def test_launch_list_totals_and_shares(tmp_path):
    f = tmp_path / "launches.csv"
    f.write_text("==PROF== Connected to process 1\n" + HEAD
                 + _row(0, "void msrsb::smooth_kernel<float, 8>(int, const int *)", "usecond", "12.5")
                 + _row(1, "void msrsb::smooth_kernel<float, 8>(int, const int *)", "nsecond", "12,500")
                 + _row(2, "msrsb::gemv_kernel(int, const double *, const double *, double *, float *)", "ns", "75000"))
    out = S.launches(str(f))
    assert out.startswith("launches 3, total 100.0 us")
    lines = [l for l in out.splitlines() if l.startswith("| `")]
    # sorted by total time: gemv 75 us (75%), then two smoothing launches 25 us (25%)
    assert lines[0] == "| `msrsb::gemv_kernel` | 1 | 75.0 | 75.00 | 75.00% |"
    assert lines[1] == "| `msrsb::smooth_kernel<float, 8>` | 2 | 25.0 | 12.50 | 25.00% |"


def test_raw_page_table(tmp_path):
    f = tmp_path / "raw.csv"
    f.write_text('"ID","Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum"\n'
                 '"","","us","Mbyte","Kbyte"\n'
                 '"0","void msrsb::smooth_kernel<float, 8>(int)","20.7","40.15","106.75"\n')
    out = S.raw(str(f))
    assert "### `msrsb::smooth_kernel<float, 8>`" in out
    assert "| dram__bytes_read.sum | 40.15 | Mbyte |" in out
    assert "| dram__bytes_write.sum | 106.75 | Kbyte |" in out
    assert "| gpu__time_duration.sum | 20.7 | us |" in out
