// Serving: a device-resident request loop with continuous batching.
//
// dpgmg_submit() queues a solve (mesh, p, omega, wavespeed, source, options)
// and returns a ticket at once.  Worker slots, each with its own CUDA stream,
// take queued requests first-fit by device memory: a request is admitted as
// soon as a slot is free and its footprint estimate fits the memory not held
// by running requests, so requests that arrive while others are on the GPU
// start as slots and memory free up, and their kernels overlap on the device.
// A request whose footprint exceeds the whole serving budget is refused at
// submission with DPGMG_ERR_NOMEM.  Each admitted request builds its own
// hierarchy on the device (Sec. 2-3), runs MG-PCG and field recovery, copies
// its trace and field solution to host memory and releases its device memory;
// dpgmg_poll() returns DPGMG_ERR_PENDING until then.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "internal.h"

namespace dpgmg {

struct Request {
  long long id = 0;
  dpgmg_problem pb{};
  dpgmg_opts op{};
  std::vector<double> ws, mf, u0;
  size_t est = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  int status = DPGMG_OK;
  std::string msg;
  std::vector<double2> trace, fields;
  dpgmg_stats st{};
};

struct Server {
  int device = 0;
  int slots = 0;
  dpgmg_handle owner = nullptr;   // its ledger admits requests (h.used + h.serving <= h.budget)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<long long, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  bool stop = false;
  long long next_id = 1;
};

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void run_request(Request& rq, cudaStream_t st, size_t budget) {
  SystemImpl S;
  try {
    dpgmg_problem pb = rq.pb;
    pb.wavespeed = rq.ws.empty() ? nullptr : rq.ws.data();
    pb.mf_coeffs = rq.mf.empty() ? nullptr : rq.mf.data();
    pb.u0_samples = rq.u0.empty() ? nullptr : rq.u0.data();
    setup_system(S, &pb, &rq.op, budget, st);
    const int64_t n = S.levels.back().mesh.ndof;
    const int64_t nf = S.nelem * S.nf;
    double2* x = S.mem.arr<double2>((size_t)n);
    double2* f = S.mem.arr<double2>((size_t)std::max<int64_t>(nf, 1));
    rq.status = pcg_solve(S, st, x, &rq.st);
    recover_fields(S, x, f, st);
    rq.trace.resize(n);
    rq.fields.resize(nf);
    DPG_CUDA(cudaMemcpyAsync(rq.trace.data(), x, (size_t)n * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DPG_CUDA(cudaMemcpyAsync(rq.fields.data(), f, (size_t)nf * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DPG_CUDA(cudaStreamSynchronize(st));
  } catch (const Err& e) {
    rq.status = e.code;
    rq.msg = e.msg;
    cudaStreamSynchronize(st);
  }
  profile_clear(S);
  free_workspace(S);
  S.mem.free_all();
  S.mem_aux.free_all();
  cudaStreamSynchronize(st);
  if (S.aux) cudaStreamSynchronize(S.aux);
}

static void worker_loop(Server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  for (;;) {
    std::shared_ptr<Request> rq;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop) break;
        {
          // first fit against the handle's ledger: set-up systems and running requests
          std::lock_guard<std::mutex> lg(sv->owner->ledger);
          HandleImpl& H = sv->owner->h;
          for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
            if ((*it)->est + H.serving + H.used <= H.budget) {
              rq = *it;
              sv->queue.erase(it);
              H.serving += rq->est;
              break;
            }
          }
        }
        if (rq) break;
        sv->cv.wait(lk);
      }
      if (!rq) break;
      rq->state = 1;
      rq->t_start = now_ms();
    }
    run_request(*rq, st, rq->est);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      {
        std::lock_guard<std::mutex> lg(sv->owner->ledger);
        sv->owner->h.serving -= std::min(sv->owner->h.serving, rq->est);
      }
      rq->t_done = now_ms();
      rq->state = 2;
    }
    sv->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

static Server* server_of(dpgmg_handle h, int slots) {
  if (!h->server) {
    auto* sv = new Server();
    sv->device = h->h.device;
    sv->slots = slots > 0 ? slots : 4;
    sv->owner = h;
    for (int i = 0; i < sv->slots; ++i) sv->workers.emplace_back(worker_loop, sv);
    h->server = sv;
  }
  return h->server;
}

void server_notify(dpgmg_handle h) {
  Server* sv = h ? h->server : nullptr;
  if (!sv) return;
  { std::lock_guard<std::mutex> lk(sv->mu); }
  sv->cv.notify_all();
}

void server_shutdown(dpgmg_handle h) {
  Server* sv = h->server;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  delete sv;
  h->server = nullptr;
}

}  // namespace dpgmg

using namespace dpgmg;

extern "C" {

int dpgmg_serve_start(dpgmg_handle h, int slots) {
  if (!h || slots < 1 || slots > 64) return DPGMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->server) return h->server->slots == slots ? DPGMG_OK : DPGMG_ERR_ARG;
  server_of(h, slots);
  return DPGMG_OK;
}

int dpgmg_submit(dpgmg_handle h, const dpgmg_problem* pb, const dpgmg_opts* op, dpgmg_ticket* ticket) {
  if (!h || !ticket) return DPGMG_ERR_ARG;
  *ticket = 0;
  int v = validate_problem(pb, op);
  if (v) {
    set_last_error("invalid problem or options");
    return v;
  }
  Server* sv;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    sv = server_of(h, 0);
  }
  auto rq = std::make_shared<Request>();
  rq->pb = *pb;
  rq->op = *op;
  const int64_t ne = (int64_t)pb->n[0] * pb->n[1] * pb->n[2];
  if (pb->wavespeed) rq->ws.assign(pb->wavespeed, pb->wavespeed + ne);
  if (pb->source == DPGMG_SRC_MANUFACTURED) {
    size_t m = pb->mf_order;
    rq->mf.assign(pb->mf_coeffs, pb->mf_coeffs + 2 * 4 * m * m * m);
  }
  if (pb->u0_samples) rq->u0.assign(pb->u0_samples, pb->u0_samples + 2 * boundary_point_count(pb));
  rq->pb.wavespeed = nullptr;
  rq->pb.mf_coeffs = nullptr;
  rq->pb.u0_samples = nullptr;
  rq->est = estimate_bytes(pb, op);
  if (rq->est > h->h.budget) {
    set_last_error("request footprint exceeds the handle's memory budget");
    return DPGMG_ERR_NOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    rq->id = sv->next_id++;
    rq->t_submit = now_ms();
    sv->all[rq->id] = rq;
    sv->queue.push_back(rq);
  }
  sv->cv.notify_all();
  *ticket = rq->id;
  return DPGMG_OK;
}

int dpgmg_poll(dpgmg_handle h, dpgmg_ticket ticket, void* trace_out, void* field_out, dpgmg_stats* st,
               double* latency_ms) {
  if (!h || !h->server) return DPGMG_ERR_ARG;
  Server* sv = h->server;
  std::shared_ptr<Request> rq;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return DPGMG_ERR_ARG;
    if (it->second->state != 2) return DPGMG_ERR_PENDING;
    rq = it->second;
    sv->all.erase(it);
  }
  if (trace_out && !rq->trace.empty())
    std::memcpy(trace_out, rq->trace.data(), rq->trace.size() * sizeof(double2));
  if (field_out && !rq->fields.empty())
    std::memcpy(field_out, rq->fields.data(), rq->fields.size() * sizeof(double2));
  if (st) {
    *st = rq->st;
    st->t_setup_ms = rq->st.t_setup_ms;
  }
  if (latency_ms) *latency_ms = rq->t_done - rq->t_submit;
  if (rq->status != DPGMG_OK) set_last_error(rq->msg.empty() ? dpgmg_strerror(rq->status) : rq->msg);
  return rq->status;
}

}  // extern "C"
